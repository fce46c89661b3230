// Split-precision radix-16 DFT on tensor cores (warp-level mma.sync
// m16n8k16, FP32 accumulation), for 32 DFT instances per warp.
//
// A complex 16-point DFT y = W x is the real 32x32 product
//   [y_re y_im] = [x_re x_im] [[Re W, Im W], [-Im W, Re W]]   (row vectors),
// i.e. Y (32 instances x 32) = X (32 x 32) Wr (32 x 32), computed as two
// 16-row M tiles x two 16-deep K steps x four 8-wide N tiles.  Operands are
// split into 16-bit hi + lo parts, x = x_hi + x_lo, W = W_hi + W_lo, and
//   Y ~ X_hi W_hi + X_hi W_lo + X_lo W_hi
// (the lo*lo term is below the FP32 accumulation error).  FP16 parts keep
// ~22 significant bits, BF16 parts ~16.  PREC 3 splits both operands into
// three BF16 parts (hi + mid + lo, ~24 significant bits) and keeps the six
// products whose order is at most 2^-16 of the leading one:
//   Y ~ Xh Wh + (Xh Wm + Xm Wh) + (Xh Wl + Xl Wh + Xm Wm),
// dropping Xm Wl, Xl Wm and Xl Wl (order 2^-24 and below).
//
// FP16 has a narrow exponent range: a small operand's lo part would fall
// into the subnormals and lose bits, a large one would overflow.  Each DFT
// instance (row of X) is therefore scaled by a power of two that brings its
// largest component into [2^14, 2^15) before the split and scaled back after
// the product (block floating point per instance; both scalings are exact).
// BF16 has FP32's exponent range and is used unscaled.
//
// Fragment ownership (lane = 4 g + tig): in the m16n8k16 layouts a lane holds
// rows g and g+8 of each M tile, at inputs k = tig, tig+4 (K step 0) and
// tig+8, tig+12 (K step 1), and returns the same rows at outputs
// n = tig + 4j, j = 0..3.  With instance mi = 2 t + h meaning warp row
// 16 t + 8 h + g, x[mi][kk] is input k = tig + 4 kk and y[mi][j] output
// n = tig + 4 j.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "conv_fft.cuh"

namespace fdas {

// The lane's four instances inside its warp: warp row 16 (mi >> 1) + 8 (mi & 1) + g,
// returned as CTA thread numbers (the instance a thread owns in the FP32 form).
struct MmaLane {
    int lane, g, tig, wbase;
    __device__ explicit MmaLane(int t) : lane(t & 31), g((t & 31) >> 2), tig(t & 3), wbase(t & ~31) {}
    __device__ __forceinline__ int inst(int mi) const {
        return wbase + 16 * (mi >> 1) + 8 * (mi & 1) + g;
    }
};

template <int PREC>   // 1 = FP16 hi+lo, 2 = BF16 hi+lo, 3 = BF16 hi+mid+lo
struct SplitMMA {
    static constexpr int NP = PREC == 3 ? 3 : 2;   // parts per operand
    uint32_t bh[2][4][2];   // [K step][N tile][reg] hi part of Wr
    uint32_t bl[2][4][2];   // lo part (PREC 3: the middle part)
    uint32_t bx[PREC == 3 ? 2 : 1][4][2];   // PREC 3: the lo part

    __device__ __forceinline__ static uint32_t pack(float a, float b) {
        if constexpr (PREC == 1) {
            __half2 h = __floats2half2_rn(a, b);
            return *reinterpret_cast<uint32_t*>(&h);
        } else {
            __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            return *reinterpret_cast<uint32_t*>(&h);
        }
    }
    __device__ __forceinline__ static float2 unpack(uint32_t u) {
        if constexpr (PREC == 1) {
            return __half22float2(*reinterpret_cast<__half2*>(&u));
        } else {
            return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&u));
        }
    }
    // hi and lo packed pairs of (a, b)
    __device__ __forceinline__ static void split(float a, float b, uint32_t& hi, uint32_t& lo) {
        hi = pack(a, b);
        const float2 h = unpack(hi);
        lo = pack(a - h.x, b - h.y);
    }
    // hi, mid and lo packed pairs of (a, b): each part rounds the remainder
    // of the parts before it
    __device__ __forceinline__ static void split3(float a, float b, uint32_t& hi, uint32_t& mid,
                                                  uint32_t& lo) {
        hi = pack(a, b);
        const float2 h = unpack(hi);
        const float ra = a - h.x, rb = b - h.y;
        mid = pack(ra, rb);
        const float2 m = unpack(mid);
        lo = pack(ra - m.x, rb - m.y);
    }

    // S = -1 forward, +1 inverse
    template <int S>
    __device__ void init(int lane) {
        const int g = lane >> 2, tig = lane & 3;
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int k = 8 * s + tig + 4 * r;      // input index of rows 2tig, 2tig+1 (+8)
                    const int n = 4 * j + (g >> 1);          // output index of column g
                    float sn, cs;
                    sincospif(2.0f * (float)((k * n) & 15) / 16.0f, &sn, &cs);
                    sn *= (float)S;
                    // column n' = 2n (re out): (Re w, -Im w); n' = 2n+1 (im out): (Im w, Re w)
                    const float w0 = (g & 1) ? sn : cs;
                    const float w1 = (g & 1) ? cs : -sn;
                    if constexpr (PREC == 3) split3(w0, w1, bh[s][j][r], bl[s][j][r], bx[s][j][r]);
                    else split(w0, w1, bh[s][j][r], bl[s][j][r]);
                }
    }

    __device__ __forceinline__ static void mma(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
        if constexpr (PREC == 1) {
            asm(
                "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                "{%8,%9}, {%0,%1,%2,%3};"
                : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
        } else {
            asm(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                "{%8,%9}, {%0,%1,%2,%3};"
                : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
        }
    }

    // Power-of-two scales (into, out of the product) of the instance whose
    // components this lane holds in x[kk]; the four lanes tig = 0..3 of the
    // instance agree on them.
    __device__ __forceinline__ static void row_scale(const float2 (&x)[4], float& sin_,
                                                     float& sout) {
        uint32_t m = 0;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            m = max(m, __float_as_uint(x[kk].x) & 0x7fffffffu);
            m = max(m, __float_as_uint(x[kk].y) & 0x7fffffffu);
        }
        m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
        // largest component in [2^(e-127), 2^(e-126)); bring it to [2^14, 2^15)
        const int e = (int)(m >> 23);
        const int k = min(max(141 - e, -100), 100);
        sin_ = __uint_as_float((uint32_t)(127 + k) << 23);
        sout = __uint_as_float((uint32_t)(127 - k) << 23);
    }

    // y[mi][j] = sum_kk W(n = tig + 4j, k = tig + 4kk) x[mi][kk] over the whole warp's rows
    __device__ void apply(const float2 (&x)[4][4], float2 (&y)[4][4]) const {
        float si[4], so[4];
#pragma unroll
        for (int mi = 0; mi < 4; ++mi) {
            if constexpr (PREC == 1) {
                row_scale(x[mi], si[mi], so[mi]);
            } else {
                si[mi] = 1.f;
                so[mi] = 1.f;
            }
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            float acc[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
            const float s0 = si[2 * t], s1 = si[2 * t + 1];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                uint32_t ah[4], al[4];
                if constexpr (PREC == 3) {
                    uint32_t ax[4];   // lo parts; al holds the middle parts
                    split3(x[2 * t][2 * s].x, x[2 * t][2 * s].y, ah[0], al[0], ax[0]);
                    split3(x[2 * t + 1][2 * s].x, x[2 * t + 1][2 * s].y, ah[1], al[1], ax[1]);
                    split3(x[2 * t][2 * s + 1].x, x[2 * t][2 * s + 1].y, ah[2], al[2], ax[2]);
                    split3(x[2 * t + 1][2 * s + 1].x, x[2 * t + 1][2 * s + 1].y, ah[3], al[3],
                           ax[3]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {   // smallest terms first
                        mma(acc[j], ah, bx[s][j]);
                        mma(acc[j], ax, bh[s][j]);
                        mma(acc[j], al, bl[s][j]);
                        mma(acc[j], ah, bl[s][j]);
                        mma(acc[j], al, bh[s][j]);
                        mma(acc[j], ah, bh[s][j]);
                    }
                } else {
                    // a0: row g, k = 8s+tig; a1: row g+8; a2: row g, k+4; a3: row g+8, k+4
                    split(x[2 * t][2 * s].x * s0, x[2 * t][2 * s].y * s0, ah[0], al[0]);
                    split(x[2 * t + 1][2 * s].x * s1, x[2 * t + 1][2 * s].y * s1, ah[1], al[1]);
                    split(x[2 * t][2 * s + 1].x * s0, x[2 * t][2 * s + 1].y * s0, ah[2], al[2]);
                    split(x[2 * t + 1][2 * s + 1].x * s1, x[2 * t + 1][2 * s + 1].y * s1, ah[3],
                          al[3]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        mma(acc[j], ah, bh[s][j]);
                        mma(acc[j], ah, bl[s][j]);
                        mma(acc[j], al, bh[s][j]);
                    }
                }
            }
            const float o0 = so[2 * t], o1 = so[2 * t + 1];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                y[2 * t][j] = make_float2(acc[j][0] * o0, acc[j][1] * o0);
                y[2 * t + 1][j] = make_float2(acc[j][2] * o1, acc[j][3] * o1);
            }
        }
    }
};

// forward_fft_d3 (conv_fft.cuh) with its two radix-16 passes on tensor cores:
// loads the L bins spec[base + p] (zero outside [0, nb)) itself, in the MMA
// instance layout, and leaves the digit-reversed spectrum in v (D3).  The
// radix-Q pass and the twiddles stay FP32.  Ends without a CTA barrier.
template <int L, int PREC>
__device__ void forward_fft_d3_split(const float2* __restrict__ spec, int64_t nb, int64_t base,
                                     float2* v, float2* buf0, float2* buf1, int t) {
    using S = ConvShape<L>;
    constexpr int T = S::T, Q = S::Q, G = S::G;
    const MmaLane ml(t);
    SplitMMA<PREC> fw;
    fw.template init<-1>(ml.lane);
    float2 xm[4][4], ym[4][4];
    // pass 1: instance = position mod T, input = digit n0 of p = n0*T + inst
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int64_t pos = base + (int64_t)(ml.tig + 4 * kk) * T + ml.inst(mi);
            xm[mi][kk] = (pos >= 0 && pos < nb) ? __ldg(&spec[pos]) : make_float2(0.f, 0.f);
        }
    fw.apply(xm, ym);
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int tm = ml.inst(mi);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k0 = ml.tig + 4 * j;
            buf0[k0 * (T + Q) + tm] = cmul(ym[mi][j], fwd_twiddle(tm * k0, L));
        }
    }
    __syncthreads();
    // pass 2: instance (a, c), input b at a*(T+Q) + b*Q + c
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int tm = ml.inst(mi);
        const float2* xb = buf0 + (tm / Q) * (T + Q) + tm % Q;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) xm[mi][kk] = xb[(ml.tig + 4 * kk) * Q];
    }
    fw.apply(xm, ym);
#pragma unroll
    for (int mi = 0; mi < 4; ++mi) {
        const int tm = ml.inst(mi), cm = tm % Q;
        float2* x2 = buf1 + (tm / Q) * G + cm;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k1 = ml.tig + 4 * j;
            x2[k1 * (Q + 1)] = cmul(ym[mi][j], fwd_twiddle((cm * k1) % (L / 16), L / 16));
        }
    }
    __syncwarp();
    const int a = t / Q, c = t % Q;
    const float2* x2 = buf1 + a * G;
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = x2[(c + Q * (i / Q)) * (Q + 1) + (i % Q)];
#pragma unroll
    for (int s2 = 0; s2 < S::NS; ++s2) dftq<Q, -1>(v + s2 * Q);
}

}  // namespace fdas
