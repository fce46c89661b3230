// Template response of a constant-fdot signal and its derivatives, shared
// by the template-bank generator and the candidate refinement.
//
// R_z(d) = int_0^1 exp(i 2 pi (z u^2/2 - (d + z/2) u)) du   (Section 2, Eqs. 22-23)
//
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
// evaluated.  For |x| < 2 the power series of F is used (FP64).  z < 0
// follows from R_{-z}(d) = e^{-i 2 pi d} conj(R_z(d)).
//
// Derivatives (candidate refinement), with moments M_n = int u^n e^{i phi}:
//   dR/dd = -i 2 pi M_1,  dR/dz = i pi (M_2 - M_1),  and, from integrating
//   phi'(u) e^{i phi} and u phi'(u) e^{i phi} by parts (z != 0),
//   M_1 = [(d + z/2) M_0 - (i/2pi)(e^{-i 2 pi d} - 1)] / z,
//   M_2 = [(d + z/2) M_1 + (i/2pi)(M_0 - e^{-i 2 pi d})] / z.
// For |z| < 1/2 these recurrences lose digits, and R and its derivatives come
// from the Taylor series in z of e^{i pi z (u^2 - u)} instead.
#pragma once
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
static __constant__ double kSerC[kSerTerms] = {
    ser_c(0), ser_c(1), ser_c(2), ser_c(3), ser_c(4), ser_c(5), ser_c(6), ser_c(7),
    ser_c(8), ser_c(9), ser_c(10), ser_c(11), ser_c(12), ser_c(13), ser_c(14), ser_c(15),
    ser_c(16), ser_c(17), ser_c(18), ser_c(19), ser_c(20), ser_c(21), ser_c(22), ser_c(23)};
static __constant__ double kSerS[kSerTerms] = {
    ser_s(0), ser_s(1), ser_s(2), ser_s(3), ser_s(4), ser_s(5), ser_s(6), ser_s(7),
    ser_s(8), ser_s(9), ser_s(10), ser_s(11), ser_s(12), ser_s(13), ser_s(14), ser_s(15),
    ser_s(16), ser_s(17), ser_s(18), ser_s(19), ser_s(20), ser_s(21), ser_s(22), ser_s(23)};

// F(x) = C(x) + i S(x) for |x| < 2 (FP64 Horner in x^4).
__device__ inline cd fresnel_series(double x) {
    const double x2 = x * x, x4 = x2 * x2;
    double c = kSerC[kSerTerms - 1], s = kSerS[kSerTerms - 1];
#pragma unroll
    for (int n = kSerTerms - 2; n >= 0; --n) {
        c = fma(c, x4, kSerC[n]);
        s = fma(s, x4, kSerS[n]);
    }
    return {x * c, x * x2 * s};
}

// Number of continued-fraction terms giving ~1e-16 for every x >= 2.
__device__ __forceinline__ int cf_terms(double x) {
    return x < 2.5 ? 48 : x < 3.2 ? 32 : x < 4.0 ? 24 : x < 5.0 ? 16 : x < 6.0 ? 12 : x < 8.0 ? 10 : 8;
}

// E(x), x >= 2, by the continued fraction evaluated from its tail.  With
// Real = float (the template bank): |E| <= 0.16 and varies slowly, and the
// FP32 evaluation is within 3e-7 of it relative, below the FP32 rounding of
// the stored taps; only the quadratic phases, which grow with |z|, need FP64.
// With Real = double (candidate refinement, where P is differentiated
// numerically and must be smooth to ~1e-12), everything is FP64.
template <typename Real>
__device__ cd fresnel_tail_e(double xd) {
    const Real x = (Real)xd;
    const Real sp2 = (Real)0.88622692545275801;   // sqrt(pi)/2
    const Real wx = sp2 * x, wy = -sp2 * x;
    const int N = cf_terms(xd);
    Real fx = wx, fy = wy;
    for (int n = N; n >= 1; --n) {
        const Real h = ((Real)0.5 * (Real)n) / (fx * fx + fy * fy);
        fx = h * fx + wx;                        // w + (n/2) conj(f)/|f|^2
        fy = -h * fy + wy;
    }
    const Real inv = (Real)1 / (fx * fx + fy * fy);
    const Real rx = fx * inv, ry = -fy * inv;
    const Real k = (Real)0.28209479177387814;     // 1/(2 sqrt(pi)); E = k (1+i) / f
    return {(double)(k * (rx - ry)), (double)(k * (rx + ry))};
}

// e^{-i pi q^2/z} F(x) for x = X (isY = 0) or x = Y (isY = 1), using the
// phase identities above for |x| >= 2.  eyd = e^{-i 2 pi d}.
template <typename Real>
__device__ cd phased_f(double x, int isY, cd ph, cd eyd) {
    const double ax = fabs(x);
    if (ax < 2.0) return cmuld(ph, fresnel_series(x));
    const double sg = x < 0 ? -1.0 : 1.0;
    cd e = fresnel_tail_e<Real>(ax);
    if (isY) e = cmuld(e, eyd);
    const cd half = cmuld(ph, cd{0.5, 0.5});
    return cscale(csub(half, e), sg);
}

// R_z(d), z > 0; eyd = e^{-i 2 pi d}.
template <typename Real>
__device__ cd response_pos(double z, double d, cd eyd) {
    const double q = -(d + 0.5 * z);
    const double s = sqrt(2.0 * z);
    const double X = s * q / z;
    const double Y = s * (1.0 + q / z);
    const cd ph = expipi(-(q * q / z));
    const cd r = csub(phased_f<Real>(Y, 1, ph, eyd), phased_f<Real>(X, 0, ph, eyd));
    return cscale(r, 1.0 / s);
}

// R_z(d) for any real z and d (the bank uses integer z and d).
template <typename Real>
__device__ cd response(double z, double d) {
    const cd eyd = (d == floor(d)) ? cd{1.0, 0.0} : expipi(-2.0 * d);
    if (z == 0.0) {
        // e^{-i pi d} sinc(d)
        if (d == 0.0) return {1.0, 0.0};
        const double m = sinpi(d) / (M_PI * d);
        return cscale(expipi(-d), m);
    }
    if (z > 0.0) return response_pos<Real>(z, d, eyd);
    cd r = response_pos<Real>(-z, d, eyd);
    r.y = -r.y;
    return cmuld(eyd, r);
}

// ---- derivatives ----------------------------------------------------------

// I_p(a) = int_0^1 u^p e^{-i a u} du for p = 0..P-1: the power series for
// |a| < 8 (terms below 1e-18 after 70), upward recurrence
// I_p = (p I_{p-1} - e^{-ia}) / (i a) otherwise (growth below 20 for p < 24).
template <int P>
__device__ void exp_moments(double a, cd* I) {
    if (fabs(a) < 8.0) {
        cd c[70];
        c[0] = {1.0, 0.0};
        for (int j = 1; j < 70; ++j) c[j] = cscale(cmuld(c[j - 1], cd{0.0, -a}), 1.0 / j);
        for (int p = 0; p < P; ++p) {
            cd s = {0.0, 0.0};
            for (int j = 69; j >= 0; --j) s = cadd(s, cscale(c[j], 1.0 / (p + j + 1)));
            I[p] = s;
        }
        return;
    }
    const cd e = expipi(-a / M_PI);
    const double ia = 1.0 / a;                       // 1/(i a) = -i / a
    // I_0 = (1 - e^{-ia}) / (i a)
    cd t = {1.0 - e.x, -e.y};
    I[0] = {t.y * ia, -t.x * ia};
    for (int p = 1; p < P; ++p) {
        t = {p * I[p - 1].x - e.x, p * I[p - 1].y - e.y};
        I[p] = {t.y * ia, -t.x * ia};
    }
}

// R, dR/dd, dR/dz for |z| < 1/2 from the Taylor series in z (10 terms:
// |pi z (u^2 - u)| <= pi/8, remainder below 3e-11):
//   R = sum_n (i pi z)^n / n! J_n,  J_n = int (u^2 - u)^n e^{-i 2 pi d u} du,
//   dR/dd = sum_n (i pi z)^n / n! (-i 2 pi) int u (u^2 - u)^n e^{..},
//   dR/dz = sum_{n>=1} i pi (i pi z)^{n-1} / (n-1)! J_n.
__device__ inline void response_derivs_small_z(double z, double d, cd& R, cd& Rd, cd& Rz) {
    constexpr int N = 10;
    cd I[2 * N + 2];
    exp_moments<2 * N + 2>(2.0 * M_PI * d, I);
    R = {0.0, 0.0};
    Rd = {0.0, 0.0};
    Rz = {0.0, 0.0};
    cd c = {1.0, 0.0};                 // (i pi z)^n / n!
    cd cprev = {0.0, 0.0};             // (i pi z)^(n-1) / (n-1)!
    for (int n = 0; n <= N; ++n) {
        // J_n = sum_k C(n,k) (-1)^{n-k} I_{n+k}, likewise with I_{n+k+1}
        cd J = {0.0, 0.0}, Ju = {0.0, 0.0};
        double binom = 1.0;
        for (int k = 0; k <= n; ++k) {
            const double sg = ((n - k) & 1) ? -binom : binom;
            J = cadd(J, cscale(I[n + k], sg));
            Ju = cadd(Ju, cscale(I[n + k + 1], sg));
            binom = binom * (n - k) / (k + 1);
        }
        R = cadd(R, cmuld(c, J));
        Rd = cadd(Rd, cmuld(c, cmuld(cd{0.0, -2.0 * M_PI}, Ju)));
        if (n >= 1) Rz = cadd(Rz, cmuld(cmuld(cd{0.0, M_PI}, cprev), J));
        cprev = c;
        c = cscale(cmuld(c, cd{0.0, M_PI * z}), 1.0 / (n + 1));
    }
}

// R_z(d), dR/dd, dR/dz in FP64 for real z and d.
__device__ inline void response_derivs(double z, double d, cd& R, cd& Rd, cd& Rz) {
    if (fabs(z) < 0.5) {
        response_derivs_small_z(z, d, R, Rd, Rz);
        return;
    }
    const cd e = expipi(-2.0 * d);                  // e^{-i 2 pi d}
    const cd M0 = response<double>(z, d);
    const double w = d + 0.5 * z, iz = 1.0 / z, k = 0.5 / M_PI;
    // M1 = [w M0 - (i/2pi)(e - 1)] / z
    const cd a1 = {w * M0.x + k * e.y, w * M0.y - k * (e.x - 1.0)};
    const cd M1 = cscale(a1, iz);
    // M2 = [w M1 + (i/2pi)(M0 - e)] / z
    const cd a2 = {w * M1.x - k * (M0.y - e.y), w * M1.y + k * (M0.x - e.x)};
    const cd M2 = cscale(a2, iz);
    R = M0;
    Rd = {2.0 * M_PI * M1.y, -2.0 * M_PI * M1.x};   // -i 2 pi M1
    Rz = {-M_PI * (M2.y - M1.y), M_PI * (M2.x - M1.x)};   // i pi (M2 - M1)
}

}  // namespace fdas
