// Register-resident small DFTs (radix 2/4/8/16/32) used by the convolver and
// the front end.  S = -1 is the forward transform  X_k = sum_n x_n e^{-i2pi nk/N},
// S = +1 the inverse without 1/N  (DFT and IDFT of Section 4.2).  Inputs and
// outputs are in natural order; all indices are compile-time constants so
// the permutations are register renames.
//
// A complex value is a float2 (re, im) in an aligned register pair, so a
// complex addition is one packed FADD2 (sm_100+), the same IEEE addition per
// component.  Products by +-i are folded into the additions that consume
// them as packed additions of the swapped, sign-flipped pair (measured: fewer
// instructions than two scalar additions), and products by constant
// twiddles are two packed operations (cmul_k).
#pragma once
#include <cuda_runtime.h>

namespace fdas {

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// (S i) * v
template <int S>
__device__ __forceinline__ float2 mul_si(float2 v) {
    return S > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}
// a + S i b  and  a - S i b
template <int S>
__device__ __forceinline__ float2 add_si(float2 a, float2 b) {
    return __fadd2_rn(a, S > 0 ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x));
}
template <int S>
__device__ __forceinline__ float2 sub_si(float2 a, float2 b) {
    return __fadd2_rn(a, S > 0 ? make_float2(b.y, -b.x) : make_float2(-b.y, b.x));
}

constexpr float kC8 = 0.92387953251128674f;  // cos(pi/8)
constexpr float kS8 = 0.38268343236508978f;  // sin(pi/8)
constexpr float kR2 = 0.70710678118654752f;  // 1/sqrt(2)

// v * (c + i s) for compile-time c, s as two packed operations:
// (v.x c, v.y c) + (v.y, v.x) (-s, s)  (the swapped pair is an operand form of
// the packed multiply-add, no extra instruction)
__device__ __forceinline__ float2 cmul_k(float2 v, float c, float s) {
    return __ffma2_rn(make_float2(v.y, v.x), make_float2(-s, s), __fmul2_rn(v, make_float2(c, c)));
}

// v * w16^m,  w16 = exp(S i 2 pi / 16),  m a compile-time constant
template <int S, int MM>
__device__ __forceinline__ float2 w16(float2 v) {
    constexpr int m = ((MM % 16) + 16) % 16;
    constexpr float sg = (float)S;
    if constexpr (m == 0) {
        return v;
    } else if constexpr (m == 4) {
        return mul_si<S>(v);
    } else if constexpr (m == 8) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (m == 12) {
        return mul_si<-S>(v);
    } else if constexpr (m == 2) {            // (1 + S i)/sqrt2
        return __fmul2_rn(add_si<S>(v, v), make_float2(kR2, kR2));
    } else if constexpr (m == 6) {            // (-1 + S i)/sqrt2
        return __fmul2_rn(sub_si<S>(v, v), make_float2(-kR2, -kR2));
    } else if constexpr (m == 10) {           // (-1 - S i)/sqrt2
        return __fmul2_rn(add_si<S>(v, v), make_float2(-kR2, -kR2));
    } else if constexpr (m == 14) {           // (1 - S i)/sqrt2
        return __fmul2_rn(sub_si<S>(v, v), make_float2(kR2, kR2));
    } else {
        // odd m: cos/sin of 2 pi m/16 from the two octant constants
        constexpr float c = (m == 1 || m == 15) ? kC8 : (m == 3 || m == 13) ? kS8
                          : (m == 5 || m == 11) ? -kS8 : -kC8;
        constexpr float s0 = (m == 1 || m == 7) ? kS8 : (m == 3 || m == 5) ? kC8
                           : (m == 9 || m == 15) ? -kS8 : -kC8;
        return cmul_k(v, c, sg * s0);
    }
}

template <int S>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a - b;
    a = a + b;
    b = t;
}

template <int S>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    const float2 s02 = x0 + x2, d02 = x0 - x2, s13 = x1 + x3, d13 = x1 - x3;
    x0 = s02 + s13;
    x2 = s02 - s13;
    x1 = add_si<S>(d02, d13);
    x3 = sub_si<S>(d02, d13);
}

// dft4 of (x0, x1, S i x2, x3): the factor on x2 folded into its additions
template <int S>
__device__ __forceinline__ void dft4_r2(float2& x0, float2& x1, float2& x2, float2& x3) {
    const float2 s02 = add_si<S>(x0, x2), d02 = sub_si<S>(x0, x2), s13 = x1 + x3, d13 = x1 - x3;
    x0 = s02 + s13;
    x2 = s02 - s13;
    x1 = add_si<S>(d02, d13);
    x3 = sub_si<S>(d02, d13);
}

// 8 points: n = 2 n1 + n2, k = k1 + 4 k2
template <int S>
__device__ __forceinline__ void dft8(float2* v) {
    dft4<S>(v[0], v[2], v[4], v[6]);
    dft4<S>(v[1], v[3], v[5], v[7]);
    v[3] = w16<S, 2>(v[3]);
    v[7] = w16<S, 6>(v[7]);
    dft2<S>(v[0], v[1]);
    dft2<S>(v[2], v[3]);
    {   // (v4, S i v5)
        const float2 t = sub_si<S>(v[4], v[5]);
        v[4] = add_si<S>(v[4], v[5]);
        v[5] = t;
    }
    dft2<S>(v[6], v[7]);
    // X[k1 + 4 k2] sits in v[2 k1 + k2]
    float2 t1 = v[1], t2 = v[2], t3 = v[3], t4 = v[4], t5 = v[5], t6 = v[6];
    v[1] = t2;
    v[2] = t4;
    v[3] = t6;
    v[4] = t1;
    v[5] = t3;
    v[6] = t5;
}

// 16 points: n = 4 n1 + n2, k = k1 + 4 k2
template <int S>
__device__ __forceinline__ void dft16(float2* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<S>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    v[5] = w16<S, 1>(v[5]);
    v[6] = w16<S, 2>(v[6]);
    v[7] = w16<S, 3>(v[7]);
    v[9] = w16<S, 2>(v[9]);
    v[11] = w16<S, 6>(v[11]);
    v[13] = w16<S, 3>(v[13]);
    v[14] = w16<S, 6>(v[14]);
    v[15] = w16<S, 9>(v[15]);
    dft4<S>(v[0], v[1], v[2], v[3]);
    dft4<S>(v[4], v[5], v[6], v[7]);
    dft4_r2<S>(v[8], v[9], v[10], v[11]);   // v[10] carries w16^4 = S i
    dft4<S>(v[12], v[13], v[14], v[15]);
    // X[k1 + 4 k2] sits in v[4 k1 + k2]: transpose the 4x4
    float2 t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int Q, int S>
__device__ __forceinline__ void dftq(float2* v) {
    if constexpr (Q == 4) {
        dft4<S>(v[0], v[1], v[2], v[3]);
    } else if constexpr (Q == 8) {
        dft8<S>(v);
    } else {
        static_assert(Q == 16, "radix");
        dft16<S>(v);
    }
}


// cos and sin of pi k / 16, k = 0..15 (for the 32-point DFT's twiddles)
constexpr float kW32c[16] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f,
                             0.83146961230254523708f, 0.70710678118654752440f,
                             0.55557023301960222474f, 0.38268343236508977173f,
                             0.19509032201612826785f, 0.0f, -0.19509032201612826785f,
                             -0.38268343236508977173f, -0.55557023301960222474f,
                             -0.70710678118654752440f, -0.83146961230254523708f,
                             -0.92387953251128675613f, -0.98078528040323044913f};
constexpr float kW32s[16] = {0.0f, 0.19509032201612826785f, 0.38268343236508977173f,
                             0.55557023301960222474f, 0.70710678118654752440f,
                             0.83146961230254523708f, 0.92387953251128675613f,
                             0.98078528040323044913f, 1.0f, 0.98078528040323044913f,
                             0.92387953251128675613f, 0.83146961230254523708f,
                             0.70710678118654752440f, 0.55557023301960222474f,
                             0.38268343236508977173f, 0.19509032201612826785f};

// v * w32^K,  w32 = exp(S i 2 pi / 32),  0 <= K < 16 a compile-time constant
template <int S, int K>
__device__ __forceinline__ float2 w32(float2 v) {
    if constexpr (K % 2 == 0) {
        return w16<S, K / 2>(v);
    } else {
        constexpr float c = kW32c[K], s = (float)S * kW32s[K];
        return cmul_k(v, c, s);
    }
}

// Last radix-2 layer of the 32-point DFT: X[K] = E[K] + w^K O[K],
// X[K+16] = E[K] - w^K O[K] for K = KK..15 (w^8 = S i folded into the adds).
template <int S, int KK>
__device__ __forceinline__ void dft32_combine(float2* v, const float2* e, const float2* o) {
    if constexpr (KK < 16) {
        if constexpr (KK == 8) {
            v[8] = add_si<S>(e[8], o[8]);
            v[24] = sub_si<S>(e[8], o[8]);
        } else {
            const float2 t = w32<S, KK>(o[KK]);
            v[KK] = e[KK] + t;
            v[KK + 16] = e[KK] - t;
        }
        dft32_combine<S, KK + 1>(v, e, o);
    }
}

// 32 points in natural order: 16-point DFTs of the even and the odd inputs,
// then one radix-2 layer.
template <int S>
__device__ __forceinline__ void dft32(float2* v) {
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    dft16<S>(e);
    dft16<S>(o);
    dft32_combine<S, 0>(v, e, o);
}

}  // namespace fdas
