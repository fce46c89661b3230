// fdas_make_templates: FP64 template responses (Fresnel integrals) and their
// L-point spectra, stored FP32 in the convolver's digit-reversed order.
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
// evaluated.  For |x| < 2 the power series of F is used.  z < 0 follows from
// R_{-z}(d) = e^{-i 2 pi d} conj(R_z(d)).
#include <math.h>

#include "internal.h"

namespace fdas {

struct cd {
    double x, y;
};
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd cmuld(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ cd cinv(cd a) {
    double n = a.x * a.x + a.y * a.y;
    return {a.x / n, -a.y / n};
}
// exp(i pi t)
__device__ __forceinline__ cd expipi(double t) {
    double s, c;
    sincospi(t, &s, &c);
    return {c, s};
}

// F(x) = int_0^x e^{i pi t^2/2} dt for |x| < 2 by its power series
//   sum_n (i pi x^2/2)^n / n! * x / (2n+1).
__device__ cd fresnel_series(double x) {
    const double a = M_PI * x * x * 0.5;
    cd p = {1.0, 0.0};
    cd s = {x, 0.0};
    for (int n = 1; n < 46; ++n) {
        p = cscale(cmuld(p, cd{0.0, a}), 1.0 / n);
        s = cadd(s, cscale(p, x / (2 * n + 1)));
    }
    return s;
}

// E(x), x >= 2: the continued fraction evaluated from the tail with a term
// count that gives ~1e-16 for every x >= 2.
__device__ cd fresnel_tail_e(double x) {
    const double sp2 = 0.88622692545275801;   // sqrt(pi)/2
    cd w = {sp2 * x, -sp2 * x};
    int N = x < 2.5 ? 48 : x < 3.2 ? 32 : x < 4.0 ? 24 : x < 5.0 ? 16 : x < 6.0 ? 12 : x < 8.0 ? 10 : 8;
    cd f = w;
    for (int n = N; n >= 1; --n) f = cadd(w, cscale(cinv(f), 0.5 * n));
    const double k = 0.28209479177387814;     // 1/(2 sqrt(pi))
    return cmuld(cd{k, k}, cinv(f));
}

// e^{-i pi q^2/z} F(x) for x = X (tag 0) or x = Y (tag 1), using the phase
// identities above for |x| >= 2.
__device__ cd phased_f(double x, int isY, double q2z, double d) {
    double ax = fabs(x);
    if (ax < 2.0) {
        cd f = fresnel_series(x);
        return cmuld(expipi(-q2z), f);
    }
    double sg = x < 0 ? -1.0 : 1.0;
    cd e = fresnel_tail_e(ax);
    if (isY) e = cmuld(e, expipi(-2.0 * d));        // e^{-i pi q^2/z} e^{i pi Y^2/2} = e^{-i 2 pi d}
    cd half = cmuld(expipi(-q2z), cd{0.5, 0.5});
    return cscale(csub(half, e), sg);
}

// R_z(d) in FP64 for integer-or-real d, z > 0.
__device__ cd response_pos(double z, double d) {
    double q = -(d + 0.5 * z);
    double s = sqrt(2.0 * z);
    double X = s * q / z;
    double Y = s * (1.0 + q / z);
    double q2z = q * q / z;
    cd fy = phased_f(Y, 1, q2z, d);
    cd fx = phased_f(X, 0, q2z, d);
    cd r = csub(fy, fx);
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

// Storage slot of frequency k in the convolver's order (see fdas.h).
__device__ __forceinline__ int bank_slot(int k, int L) {
    const int Q = L / 256, T = L / 16;
    int a = k & 15, k1 = (k >> 4) & 15, c2 = k >> 8;
    int c1 = k1 % Q, s2 = k1 / Q;
    int t = a * Q + c1, i = s2 * Q + c2;
    return 2 * ((i >> 1) * T + t) + (i & 1);
}

constexpr int kTplThreads = 512;
constexpr int kMaxTaps = 2 * 1024 + 1;

// One CTA per bank row.  Phase 1: taps conj(R_z(d)) in FP64, rounded to
// FP32 in shared memory.  Phase 2: H[k] = (1/L) sum_d conj(R(d)) e^{+i 2 pi d k/L}
// (= FFT_L of the circularly placed kernel g[j] = conj(R(-j)), over 1/L),
// accumulated in FP32 with Kahan compensation against a twiddle table.
__global__ void __launch_bounds__(kTplThreads) templates_kernel(int L, int zfirst, int zstep,
                                                                float2* __restrict__ bank) {
    extern __shared__ float2 tsm[];
    float2* tw = tsm;            // L entries: e^{+i 2 pi m / L}
    float2* taps = tsm + L;      // 2h+1 entries
    const int b = blockIdx.x;
    const int z = zfirst + b * zstep;
    const int az = z < 0 ? -z : z;
    const int h = (az + 1) / 2 + 8;
    for (int d = -h + (int)threadIdx.x; d <= h; d += blockDim.x) {
        cd r = response((double)z, (double)d);
        taps[d + h] = make_float2((float)r.x, (float)-r.y);
    }
    for (int m = threadIdx.x; m < L; m += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)m / (float)L, &s, &c);
        tw[m] = make_float2(c, s);
    }
    __syncthreads();
    const float invL = 1.0f / (float)L;
    const int mask = L - 1;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
        for (int d = -h; d <= h; ++d) {
            float2 g = taps[d + h];
            float2 w = tw[((d & mask) * k) & mask];
            float tx = fmaf(g.x, w.x, -g.y * w.y);
            float ty = fmaf(g.x, w.y, g.y * w.x);
            float yx = tx - cx, yy = ty - cy;
            float nx = sx + yx, ny = sy + yy;
            cx = (nx - sx) - yx;
            cy = (ny - sy) - yy;
            sx = nx;
            sy = ny;
        }
        bank[(size_t)b * L + bank_slot(k, L)] = make_float2(sx * invL, sy * invL);
    }
}

int launch_templates(const fdas_params* p, const Grid& g, float2* bank, cudaStream_t st) {
    if (g.hmax * 2 + 1 > kMaxTaps) return FDAS_E_UNSUPPORTED;
    size_t sm = (size_t)(p->L + 2 * g.hmax + 1) * sizeof(float2);
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(templates_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((4096 + kMaxTaps) * sizeof(float2)));
        if (e != cudaSuccess) return FDAS_E_CUDA;
        attr_done = true;
    }
    int zfirst = p->zmin + g.j0 * p->zstep;
    templates_kernel<<<g.Kb, kTplThreads, sm, st>>>(p->L, zfirst, p->zstep, bank);
    return cuda_status(cudaGetLastError());
}

}  // namespace fdas
