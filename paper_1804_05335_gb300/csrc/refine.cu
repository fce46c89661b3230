// Candidate refinement over continuous (r, z): the correlation of Eq. 23
// evaluated off the template grid, its derivatives, and gradient ascent.
// The paper recovers accurate (r, z) by fine-binning the f-fdot plane around
// a detection (Section 5.2, last paragraph); here the power is maximised
// directly:
//   S(r, z) = sum_{k=[r]-m}^{[r]+m} A_k conj(R_z(k - r)),   P = |S|^2,
//   [r] = floor(r + 1/2), A_k = 0 outside [0, nb),
//   dP/dr = 2 Re(conj(S) dS/dr),  dS/dr = -sum A_k conj(R'_d(k - r)),
//   dP/dz = 2 Re(conj(S) dS/dz),  dS/dz =  sum A_k conj(R'_z(k - r)),
//   dP/dA_k = 2 S R_z(k - r)   (d/dRe + i d/dIm).
// One warp per candidate; R and its derivatives in FP64 (fresnel.cuh).
#include "fresnel.cuh"
#include "internal.h"

namespace fdas {

constexpr int kRefThreads = 128;   // 4 candidates (warps) per CTA

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct RefSums {
    cd S, Sr, Sz;
};

// S, dS/dr, dS/dz of one candidate, summed over the warp (every lane gets them).
__device__ RefSums refine_sums(const float2* __restrict__ spec, int64_t nb, double r, double z,
                               int m, int lane) {
    const int64_t k0 = (int64_t)floor(r + 0.5);
    cd S = {0.0, 0.0}, Sr = {0.0, 0.0}, Sz = {0.0, 0.0};
    for (int i = lane; i <= 2 * m; i += 32) {
        const int64_t k = k0 - m + i;
        if (k < 0 || k >= nb) continue;
        const double d = (double)k - r;
        cd R, Rd, Rz;
        response_derivs(z, d, R, Rd, Rz);
        const float2 a = __ldg(&spec[k]);
        // A conj(R), A conj(-Rd), A conj(Rz)
        S.x += a.x * R.x + a.y * R.y;
        S.y += a.y * R.x - a.x * R.y;
        Sr.x -= a.x * Rd.x + a.y * Rd.y;
        Sr.y -= a.y * Rd.x - a.x * Rd.y;
        Sz.x += a.x * Rz.x + a.y * Rz.y;
        Sz.y += a.y * Rz.x - a.x * Rz.y;
    }
    RefSums out;
    out.S = {warp_sum(S.x), warp_sum(S.y)};
    out.Sr = {warp_sum(Sr.x), warp_sum(Sr.y)};
    out.Sz = {warp_sum(Sz.x), warp_sum(Sz.y)};
    return out;
}

__global__ void __launch_bounds__(kRefThreads) refine_fwd_kernel(
    const float2* __restrict__ spec, int64_t nb, const double* __restrict__ r,
    const double* __restrict__ z, int ncand, int m, double* __restrict__ P,
    double* __restrict__ dPdr, double* __restrict__ dPdz, double* __restrict__ Sout) {
    const int c = blockIdx.x * (kRefThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= ncand) return;
    const RefSums s = refine_sums(spec, nb, r[c], z[c], m, lane);
    if (lane == 0) {
        P[c] = s.S.x * s.S.x + s.S.y * s.S.y;
        if (dPdr) dPdr[c] = 2.0 * (s.S.x * s.Sr.x + s.S.y * s.Sr.y);
        if (dPdz) dPdz[c] = 2.0 * (s.S.x * s.Sz.x + s.S.y * s.Sz.y);
        if (Sout) {
            Sout[2 * c] = s.S.x;
            Sout[2 * c + 1] = s.S.y;
        }
    }
}

// grad_spec[k] += gP * 2 S R_z(k - r) for every tap of every candidate.
__global__ void __launch_bounds__(kRefThreads) refine_bwd_kernel(
    int64_t nb, const double* __restrict__ r, const double* __restrict__ z, int ncand, int m,
    const double* __restrict__ S, const double* __restrict__ gP, float2* __restrict__ grad_spec) {
    const int c = blockIdx.x * (kRefThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= ncand) return;
    const double rc = r[c], zc = z[c], g2 = 2.0 * gP[c];
    const cd Sc = {S[2 * c], S[2 * c + 1]};
    const int64_t k0 = (int64_t)floor(rc + 0.5);
    for (int i = lane; i <= 2 * m; i += 32) {
        const int64_t k = k0 - m + i;
        if (k < 0 || k >= nb) continue;
        const cd R = response<double>(zc, (double)k - rc);
        const cd gk = cscale(cmuld(Sc, R), g2);
        atomicAdd(&grad_spec[k].x, (float)gk.x);
        atomicAdd(&grad_spec[k].y, (float)gk.y);
    }
}

// Gradient ascent on log P, one warp per candidate, all steps in one launch:
//   r += clamp(lr_r (dP/dr)/P, +-0.5),  z += clamp(lr_z (dP/dz)/P, +-2).
__global__ void __launch_bounds__(kRefThreads) refine_ascent_kernel(
    const float2* __restrict__ spec, int64_t nb, const double* __restrict__ r_in,
    const double* __restrict__ z_in, int ncand, int m, int steps, double lr_r, double lr_z,
    double* __restrict__ r_out, double* __restrict__ z_out, double* __restrict__ P_out) {
    const int c = blockIdx.x * (kRefThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= ncand) return;
    double rc = r_in[c], zc = z_in[c], P = 0.0;
    for (int it = 0; it <= steps; ++it) {
        const RefSums s = refine_sums(spec, nb, rc, zc, m, lane);
        P = s.S.x * s.S.x + s.S.y * s.S.y;
        if (it == steps || !(P > 0.0)) break;
        const double gr = 2.0 * (s.S.x * s.Sr.x + s.S.y * s.Sr.y) / P;
        const double gz = 2.0 * (s.S.x * s.Sz.x + s.S.y * s.Sz.y) / P;
        rc += fmin(fmax(lr_r * gr, -0.5), 0.5);
        zc += fmin(fmax(lr_z * gz, -2.0), 2.0);
    }
    if (lane == 0) {
        r_out[c] = rc;
        z_out[c] = zc;
        P_out[c] = P;
    }
}

static inline unsigned ref_grid(int ncand) {
    return (unsigned)((ncand + kRefThreads / 32 - 1) / (kRefThreads / 32));
}

}  // namespace fdas

using namespace fdas;

extern "C" {

int fdas_refine_fwd(const float* spec, int64_t nb, const double* r, const double* z,
                    int32_t ncand, int32_t m, double* P, double* dPdr, double* dPdz, double* S,
                    void* stream) {
    if (!spec || !r || !z || !P || nb < 1 || ncand < 0 || m < 0 || m > 65536) return FDAS_E_INVAL;
    if (!aligned(spec, 8) || !aligned(r, 8) || !aligned(z, 8) || !aligned(P, 8)) return FDAS_E_INVAL;
    if (ncand == 0) return FDAS_OK;
    refine_fwd_kernel<<<ref_grid(ncand), kRefThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2*>(spec), nb, r, z, ncand, m, P, dPdr, dPdz, S);
    return cuda_status(cudaGetLastError());
}

int fdas_refine_bwd(const float* spec, int64_t nb, const double* r, const double* z,
                    int32_t ncand, int32_t m, const double* S, const double* gP, float* grad_spec,
                    void* stream) {
    (void)spec;
    if (!r || !z || !S || !gP || !grad_spec || nb < 1 || ncand < 0 || m < 0 || m > 65536)
        return FDAS_E_INVAL;
    if (!aligned(grad_spec, 8) || !aligned(S, 8)) return FDAS_E_INVAL;
    if (ncand == 0) return FDAS_OK;
    refine_bwd_kernel<<<ref_grid(ncand), kRefThreads, 0, (cudaStream_t)stream>>>(
        nb, r, z, ncand, m, S, gP, reinterpret_cast<float2*>(grad_spec));
    return cuda_status(cudaGetLastError());
}

int fdas_refine(const float* spec, int64_t nb, const double* r_in, const double* z_in,
                int32_t ncand, int32_t m, int32_t steps, double lr_r, double lr_z, double* r_out,
                double* z_out, double* P_out, void* stream) {
    if (!spec || !r_in || !z_in || !r_out || !z_out || !P_out || nb < 1 || ncand < 0 || m < 0 ||
        m > 65536 || steps < 0 || steps > 100000)
        return FDAS_E_INVAL;
    if (!aligned(spec, 8)) return FDAS_E_INVAL;
    if (ncand == 0) return FDAS_OK;
    refine_ascent_kernel<<<ref_grid(ncand), kRefThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2*>(spec), nb, r_in, z_in, ncand, m, steps, lr_r, lr_z,
        r_out, z_out, P_out);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
