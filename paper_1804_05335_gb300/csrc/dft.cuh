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
// a * b and a * conj(b) as two packed operations, b broadcast into the pairs
// (b.x, b.x) and (-b.y, b.y) (the warp convolver's template products and
// table twiddles; measured 3 % faster there than the scalar forms above)
__device__ __forceinline__ float2 cmul_p(float2 a, float2 b) {
    return __ffma2_rn(make_float2(a.y, a.x), make_float2(-b.y, b.y), __fmul2_rn(a, make_float2(b.x, b.x)));
}
__device__ __forceinline__ float2 cmulc_p(float2 a, float2 b) {
    return __ffma2_rn(make_float2(a.y, a.x), make_float2(b.y, -b.y), __fmul2_rn(a, make_float2(b.x, b.x)));
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

constexpr float kS3 = 0.86602540378443864676f;   // sin(pi/3) = sqrt(3)/2

// 3 points: X1,2 = a - (b + c)/2 +- S i (sqrt3/2)(b - c)
template <int S>
__device__ __forceinline__ void dft3(float2& a, float2& b, float2& c) {
    const float2 t1 = b + c;
    const float2 t2 = __ffma2_rn(t1, make_float2(-0.5f, -0.5f), a);
    const float2 d = __fmul2_rn(b - c, make_float2(kS3, kS3));
    a = a + t1;
    b = add_si<S>(t2, d);
    c = sub_si<S>(t2, d);
}

// v * w^m, w = exp(S i 2 pi / 12), m a compile-time constant
template <int S, int M>
__device__ __forceinline__ float2 w12(float2 v) {
    constexpr int m = ((M % 12) + 12) % 12;
    if constexpr (m == 0) {
        return v;
    } else if constexpr (m == 3) {
        return mul_si<S>(v);
    } else if constexpr (m == 6) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (m == 9) {
        return mul_si<-S>(v);
    } else {
        // cos and sin of 2 pi m / 12 for m = 1, 2, 4, 5, 7, 8, 10, 11
        constexpr float c = (m == 1 || m == 11) ? kS3 : (m == 2 || m == 10) ? 0.5f
                          : (m == 4 || m == 8) ? -0.5f : -kS3;
        constexpr float s0 = (m == 1 || m == 5) ? 0.5f : (m == 2 || m == 4) ? kS3
                           : (m == 7 || m == 11) ? -0.5f : -kS3;
        return cmul_k(v, c, (float)S * s0);
    }
}

// 6 points in natural order: n = 2 n1 + n2, k = k1 + 3 k2
template <int S>
__device__ __forceinline__ void dft6(float2* v) {
    dft3<S>(v[0], v[2], v[4]);
    dft3<S>(v[1], v[3], v[5]);
    const float2 e[3] = {v[0], v[2], v[4]};
    const float2 o[3] = {v[1], w12<S, 2>(v[3]), w12<S, 4>(v[5])};
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        v[k1] = e[k1] + o[k1];
        v[k1 + 3] = e[k1] - o[k1];
    }
}

// 12 points in natural order: n = 4 n1 + n2, k = k1 + 3 k2; the 3-point DFTs
// over n1, twiddles w12^(n2 k1), the 4-point DFTs over n2
template <int S>
__device__ __forceinline__ void dft12(float2* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft3<S>(v[n2], v[4 + n2], v[8 + n2]);
    // v[n2 + 4 k1] = A[n2][k1]
    float2 a[3][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) a[0][n2] = v[n2];
    a[1][0] = v[4];
    a[1][1] = w12<S, 1>(v[5]);
    a[1][2] = w12<S, 2>(v[6]);
    a[1][3] = w12<S, 3>(v[7]);
    a[2][0] = v[8];
    a[2][1] = w12<S, 2>(v[9]);
    a[2][2] = w12<S, 4>(v[10]);
    a[2][3] = w12<S, 6>(v[11]);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        dft4<S>(a[k1][0], a[k1][1], a[k1][2], a[k1][3]);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 3 * k2] = a[k1][k2];
    }
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

// Butterfly (a, b) -> (a + w b, a - w b) with the compile-time twiddle
// w = w32^K = exp(S i 2 pi K / 32), in three packed multiply-adds (the
// tangent form of the butterfly, Linzer and Feig):
//   |s| <= |c|:  w b = c u,    u = b + i (s/c) b,
//   |s| >  |c|:  w b = i s u,  u = b - i (c/s) b,
// u one multiply-add of the swapped pair, each output one more.  A product
// followed by two additions takes four packed operations.  w = +-1, +-i:
// two additions.
template <int S, int K>
__device__ __forceinline__ void bfly32(float2& a, float2& b) {
    constexpr int k = ((K % 32) + 32) % 32;
    if constexpr (k == 0) {
        const float2 t = a - b;
        a = a + b;
        b = t;
    } else if constexpr (k == 16) {
        const float2 t = a + b;
        a = a - b;
        b = t;
    } else if constexpr (k == 8) {      // w = S i
        const float2 t = sub_si<S>(a, b);
        a = add_si<S>(a, b);
        b = t;
    } else if constexpr (k == 24) {     // w = -S i
        const float2 t = add_si<S>(a, b);
        a = sub_si<S>(a, b);
        b = t;
    } else {
        constexpr float c = k < 16 ? kW32c[k] : -kW32c[k - 16];
        constexpr float s = (float)S * (k < 16 ? kW32s[k] : -kW32s[k - 16]);
        constexpr float ac = c < 0.f ? -c : c, as = s < 0.f ? -s : s;
        const float2 bs = make_float2(b.y, b.x);
        if constexpr (k % 8 == 4) {     // |c| = |s|: u = b +- i b, one addition
            const float2 u = (s / c > 0.f) ? add_si<1>(b, b) : sub_si<1>(b, b);
            const float2 x = __ffma2_rn(u, make_float2(c, c), a);
            b = __ffma2_rn(u, make_float2(-c, -c), a);
            a = x;
        } else if constexpr (as <= ac) {
            constexpr float t = s / c;
            const float2 u = __ffma2_rn(bs, make_float2(-t, t), b);
            const float2 x = __ffma2_rn(u, make_float2(c, c), a);
            b = __ffma2_rn(u, make_float2(-c, -c), a);
            a = x;
        } else {
            constexpr float ct = c / s;
            const float2 u = __ffma2_rn(bs, make_float2(ct, -ct), b);
            const float2 us = make_float2(u.y, u.x);
            const float2 x = __ffma2_rn(us, make_float2(-s, s), a);
            b = __ffma2_rn(us, make_float2(s, -s), a);
            a = x;
        }
    }
}

// 16 points (n = 4 n1 + n2, k = k1 + 4 k2) in tangent-form butterflies: the
// column DFTs over n1, then per row k1 the twiddles w16^(n2 k1) folded into
// the row DFT: with b_n2 the row's values,
//   (b0, b2) and (b1, b3) by w16^(2 k1)  -> (s02, d02), (q+, q-),
//   (s02, q+) by w16^k1, (d02, q-) by S i w16^k1  -> X0, X2, X1, X3.
// (w16^m = w32^(2m).)  74 packed operations against 80 for dft16.
template <int S, int K1>
__device__ __forceinline__ void dft16t_row(float2* b) {
    bfly32<S, 4 * K1>(b[0], b[2]);       // s02, d02
    bfly32<S, 4 * K1>(b[1], b[3]);       // q+, q-
    bfly32<S, 2 * K1>(b[0], b[1]);       // X0, X2
    bfly32<S, 2 * K1 + 8>(b[2], b[3]);   // X1, X3
    const float2 x1 = b[2], x2 = b[1];
    b[1] = x1;
    b[2] = x2;
}

template <int S>
__device__ __forceinline__ void dft16t(float2* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<S>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    dft16t_row<S, 0>(v);
    dft16t_row<S, 1>(v + 4);
    dft16t_row<S, 2>(v + 8);
    dft16t_row<S, 3>(v + 12);
    // X[k1 + 4 k2] sits in v[4 k1 + k2]: transpose the 4x4
    float2 t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int S, int K>
__device__ __forceinline__ void dft32_combine(float2* e, float2* o) {
    if constexpr (K < 16) {
        bfly32<S, K>(e[K], o[K]);
        dft32_combine<S, K + 1>(e, o);
    }
}

// 32 points in natural order: 16-point DFTs of the even and the odd inputs,
// then one radix-2 layer X[K] = E[K] + w32^K O[K], X[K + 16] = E[K] - w32^K O[K].
template <int S>
__device__ __forceinline__ void dft32(float2* v) {
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    dft16t<S>(e);
    dft16t<S>(o);
    dft32_combine<S, 0>(e, o);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = e[i];
        v[i + 16] = o[i];
    }
}

}  // namespace fdas
