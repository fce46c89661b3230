// fdas_make_templates: FP64 template responses (Fresnel integrals) and their
// L-point spectra, stored FP32 in the convolver's digit-reversed order.  The
// spectra come from the convolver's own forward FFT, so no reordering is
// ever needed (Section 4.2: the templates must be transformed by the same
// algorithm as the segments).
//
// Response of a unit constant-fdot signal at offset d from its
// mid-observation bin (Section 2, Eqs. 22-23):
//   R_z(d) = int_0^1 exp(i 2 pi (z u^2/2 - (d + z/2) u)) du.
// Completing the square with q = -(d + z/2), for z > 0,
//   R = e^{-i pi q^2/z} [F(Y) - F(X)] / sqrt(2z),
//   X = sqrt(2z) q/z,  Y = sqrt(2z)(1 + q/z),
//   F(x) = C(x) + i S(x) = int_0^x e^{i pi t^2/2} dt.
// For |x| >= 2, F(x) = sgn(x) [(1+i)/2 - e^{i pi x^2/2} E(|x|)], where
//   E(x) = (1+i)/(2 sqrt(pi)) * 1/(w + (1/2)/(w + 1/(w + (3/2)/(w + ...)))),
//   w = (sqrt(pi)/2)(1-i) x
// is the Laplace continued fraction of erfc (its tail integral).  Because
// pi X^2/2 = pi q^2/z and pi Y^2/2 - pi q^2/z = -2 pi d (mod 2 pi), the large
// quadratic phases cancel analytically and only bounded phases are ever
// evaluated.  For |x| < 2 the power series of F is used (FP64); E is
// evaluated in FP32 (bounded and smooth, see fresnel_tail_e).  z < 0 follows from
// R_{-z}(d) = e^{-i 2 pi d} conj(R_z(d)).
#include <math.h>

#include "conv_fft.cuh"
#include "internal.h"

namespace fdas {

struct cd {
    double x, y;
};
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd cmuld(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.x * s, a.y * s}; }
// exp(i pi t)
__device__ __forceinline__ cd expipi(double t) {
    double s, c;
    sincospi(t, &s, &c);
    return {c, s};
}

// Power series of the Fresnel integrals in powers of x^4, coefficients from
// their definitions:  C(x) = x sum_n (-1)^n (pi/2)^{2n} x^{4n} / ((2n)! (4n+1)),
//                     S(x) = x^3 sum_n (-1)^n (pi/2)^{2n+1} x^{4n} / ((2n+1)! (4n+3)).
constexpr double kHalfPi = 1.57079632679489662;
constexpr double cfact(int k) { return k <= 1 ? 1.0 : k * cfact(k - 1); }
constexpr double cpow(double b, int e) { return e == 0 ? 1.0 : b * cpow(b, e - 1); }
constexpr double ser_c(int n) {
    return (n % 2 ? -1.0 : 1.0) * cpow(kHalfPi, 2 * n) / (cfact(2 * n) * (4 * n + 1));
}
constexpr double ser_s(int n) {
    return (n % 2 ? -1.0 : 1.0) * cpow(kHalfPi, 2 * n + 1) / (cfact(2 * n + 1) * (4 * n + 3));
}
constexpr int kSerTerms = 24;   // |x| < 2: the last term is below 1e-22
__constant__ double kSerC[kSerTerms] = {
    ser_c(0), ser_c(1), ser_c(2), ser_c(3), ser_c(4), ser_c(5), ser_c(6), ser_c(7),
    ser_c(8), ser_c(9), ser_c(10), ser_c(11), ser_c(12), ser_c(13), ser_c(14), ser_c(15),
    ser_c(16), ser_c(17), ser_c(18), ser_c(19), ser_c(20), ser_c(21), ser_c(22), ser_c(23)};
__constant__ double kSerS[kSerTerms] = {
    ser_s(0), ser_s(1), ser_s(2), ser_s(3), ser_s(4), ser_s(5), ser_s(6), ser_s(7),
    ser_s(8), ser_s(9), ser_s(10), ser_s(11), ser_s(12), ser_s(13), ser_s(14), ser_s(15),
    ser_s(16), ser_s(17), ser_s(18), ser_s(19), ser_s(20), ser_s(21), ser_s(22), ser_s(23)};

// F(x) = C(x) + i S(x) for |x| < 2 (FP64 Horner in x^4).
__device__ cd fresnel_series(double x) {
    const double x2 = x * x, x4 = x2 * x2;
    double c = kSerC[kSerTerms - 1], s = kSerS[kSerTerms - 1];
#pragma unroll
    for (int n = kSerTerms - 2; n >= 0; --n) {
        c = fma(c, x4, kSerC[n]);
        s = fma(s, x4, kSerS[n]);
    }
    return {x * c, x * x2 * s};
}

// E(x), x >= 2, by the continued fraction evaluated from its tail, in FP32:
// |E| <= 0.16 and varies slowly, and the FP32 evaluation is within 3e-7 of
// it relative, below the FP32 rounding of the stored taps.  Only the
// quadratic phases, which grow with |z|, need FP64.
__device__ cd fresnel_tail_e(double xd) {
    const float x = (float)xd;
    const float sp2 = 0.88622692545275801f;   // sqrt(pi)/2
    const float wx = sp2 * x, wy = -sp2 * x;
    const int N = x < 2.5f ? 48 : x < 3.2f ? 32 : x < 4.0f ? 24 : x < 5.0f ? 16
                : x < 6.0f ? 12 : x < 8.0f ? 10 : 8;
    float fx = wx, fy = wy;
    for (int n = N; n >= 1; --n) {
        const float h = (0.5f * (float)n) / fmaf(fx, fx, fy * fy);
        fx = fmaf(h, fx, wx);                    // w + (n/2) conj(f)/|f|^2
        fy = fmaf(-h, fy, wy);
    }
    const float inv = 1.0f / fmaf(fx, fx, fy * fy);
    const float rx = fx * inv, ry = -fy * inv;
    const float k = 0.28209479177387814f;     // 1/(2 sqrt(pi)); E = k (1+i) / f
    return {(double)(k * (rx - ry)), (double)(k * (rx + ry))};
}

// e^{-i pi q^2/z} F(x) for x = X (isY = 0) or x = Y (isY = 1), using the
// phase identities above for |x| >= 2.  eyd = e^{-i 2 pi d}.
__device__ cd phased_f(double x, int isY, cd ph, cd eyd) {
    const double ax = fabs(x);
    if (ax < 2.0) return cmuld(ph, fresnel_series(x));
    const double sg = x < 0 ? -1.0 : 1.0;
    cd e = fresnel_tail_e(ax);
    if (isY) e = cmuld(e, eyd);
    const cd half = cmuld(ph, cd{0.5, 0.5});
    return cscale(csub(half, e), sg);
}

// R_z(d) in FP64 for integer-or-real d, z > 0.
__device__ cd response_pos(double z, double d) {
    const double q = -(d + 0.5 * z);
    const double s = sqrt(2.0 * z);
    const double X = s * q / z;
    const double Y = s * (1.0 + q / z);
    const cd ph = expipi(-(q * q / z));
    const cd eyd = (d == floor(d)) ? cd{1.0, 0.0} : expipi(-2.0 * d);
    const cd r = csub(phased_f(Y, 1, ph, eyd), phased_f(X, 0, ph, eyd));
    return cscale(r, 1.0 / s);
}

__device__ cd response(double z, double d) {
    if (z == 0.0) {
        // e^{-i pi d} sinc(d)
        if (d == 0.0) return {1.0, 0.0};
        double sn = sinpi(d);
        double m = sn / (M_PI * d);
        return cscale(expipi(-d), m);
    }
    if (z > 0.0) return response_pos(z, d);
    cd r = response_pos(-z, d);
    r.y = -r.y;
    return cmuld(expipi(-2.0 * d), r);
}

constexpr int kTapThreads = 128;

// Kernel 1: one thread per (bank row b, offset d), d = -h..h.  Writes the
// FIR kernel taps g[j] = conj(R_z(-j)) / L for j = -d to the start of bank
// row b as tap index j + h (float2), where the row-b CTA of kernel 2 reads
// them before it overwrites the row.
__global__ void __launch_bounds__(kTapThreads) template_taps_kernel(int L, int zfirst, int zstep,
                                                                    int width, int rows,
                                                                    float2* __restrict__ bank) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= rows * width) return;
    const int b = gid / width, idx = gid - b * width;
    const int z = zfirst + b * zstep;
    const int az = z < 0 ? -z : z;
    const int h = (az + 1) / 2 + 8;
    if (idx > 2 * h) return;
    const int j = idx - h;                       // tap position (circular index j mod L)
    const cd r = response((double)z, (double)(-j));
    const double s = 1.0 / (double)L;
    bank[(size_t)b * (L + 16) + idx] = make_float2((float)(r.x * s), (float)(-r.y * s));
}

// Kernel 2: one CTA of L/16 threads per bank row: gather the circularly
// placed kernel g (D1 distribution), forward FFT with the convolver's own
// permutation-free transform, store the digit-reversed spectrum in place.
template <int L>
__global__ void __launch_bounds__(L / 16) template_fft_kernel(int zfirst, int zstep,
                                                              float2* __restrict__ bank) {
    using S = ConvShape<L>;
    constexpr int T = S::T;
    extern __shared__ float4 tsm4[];
    float2* buf0 = reinterpret_cast<float2*>(tsm4);
    float2* buf1 = buf0 + S::BUFS;
    const int b = blockIdx.x, t = threadIdx.x;
    const int z = zfirst + b * zstep;
    const int az = z < 0 ? -z : z;
    const int h = (az + 1) / 2 + 8;
    float2* row = bank + (size_t)b * S::ROW;
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int p = i * T + t;
        const int j = p <= h ? p : p - L;        // circular tap position
        v[i] = (j >= -h && j <= h) ? row[j + h] : make_float2(0.f, 0.f);
    }
    __syncthreads();   // every tap is read before the row is overwritten
    forward_fft_d3<L>(v, buf0, buf1, t);
    float4* row4 = reinterpret_cast<float4*>(row);
#pragma unroll
    for (int ip = 0; ip < 8; ++ip)
        row4[ip * T + t] = make_float4(v[2 * ip].x, v[2 * ip].y, v[2 * ip + 1].x, v[2 * ip + 1].y);
    if (t == 0) {
        // mirror slots: float4 L/2 + j holds (H[-k(2ip+1)], H[-k(2ip)]) of thread 0, ip = 7 - j,
        // so that the conjugate-template read of thread 0 has the same form as everyone's
        constexpr int Q = S::Q;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ip = 7 - j;
            const float2 hi = v[thread0_mirror<Q>(2 * ip + 1)], lo = v[thread0_mirror<Q>(2 * ip)];
            row4[L / 2 + j] = make_float4(hi.x, hi.y, lo.x, lo.y);
        }
    }
}

template <int L>
static int launch_fft(int rows, int zfirst, int zstep, float2* bank, cudaStream_t st) {
    constexpr size_t sm = 2 * ConvShape<L>::BUFS * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(template_fft_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
            return FDAS_E_CUDA;
        attr = true;
    }
    template_fft_kernel<L><<<rows, L / 16, sm, st>>>(zfirst, zstep, bank);
    return cuda_status(cudaGetLastError());
}

int launch_templates(const fdas_params* p, const Grid& g, float2* bank, cudaStream_t st) {
    const int width = 2 * g.hmax + 1;
    if (width > p->L + 16) return FDAS_E_UNSUPPORTED;
    const int zfirst = p->zmin + g.j0 * p->zstep;
    const int total = g.Kb * width;
    template_taps_kernel<<<(total + kTapThreads - 1) / kTapThreads, kTapThreads, 0, st>>>(
        p->L, zfirst, p->zstep, width, g.Kb, bank);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return FDAS_E_CUDA;
    switch (p->L) {
        case 1024: return launch_fft<1024>(g.Kb, zfirst, p->zstep, bank, st);
        case 2048: return launch_fft<2048>(g.Kb, zfirst, p->zstep, bank, st);
        case 4096: return launch_fft<4096>(g.Kb, zfirst, p->zstep, bank, st);
        default: return FDAS_E_INVAL;
    }
}

}  // namespace fdas
