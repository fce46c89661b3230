// The 1024-point FFT held by one warp, used by the L = 1024 convolver and by
// the template bank generator for that length (the bank must be transformed
// by the same algorithm as the segments, Section 4.2).
//
// 1024 = 32 x 32.  Lane l holds positions p = l + 32 i in registers v[i].
// Forward (X_k = sum_p x_p W^{-pk}, W = exp(+i 2 pi / 1024), p = n1 + 32 n2):
//   1. 32-point DFT over the registers (n2 -> k1), lane n1 = l;
//   2. twiddle W^{-n1 k1};
//   3. transpose the warp's 32 x 32 matrix through shared memory, so that
//      lane k1 holds the 32 values of n1;
//   4. 32-point DFT over the registers (n1 -> k2):
//      X[k1 + 32 k2] ends in lane k1, register k2 -- natural order, the same
//      distribution as the input, k = l + 32 i.
// The inverse (no 1/L; the bank carries it) is the same sequence with
// exp(+...) in both DFTs and the twiddle W^{+n1 k2}, mapping k = l + 32 i
// back to p = l + 32 i.  One exchange per transform, inside the warp: only
// __syncwarp, never a CTA barrier.
#pragma once
#include "dft.cuh"
#include "internal.h"

namespace fdas {

struct WShape {
    static constexpr int L = 1024;
    static constexpr int NW = kWarpSegments;   // warps (one segment each) per convolver CTA
    static constexpr int NBUF = 2;          // bank rows staged per convolver CTA (measured: 2 beats 3)
    // bank row: 16 register pairs x (32 lanes + a mirror column), float4 each
    static constexpr int ROW4 = 16 * 33;
    static constexpr int XS = 34;           // exchange row stride in float2 (32 + 2 pad)
    static constexpr int XBUF = 32 * XS;    // float2 per warp exchange buffer
    static constexpr int TW4 = 16 * 32;     // float4 of the twiddle table
};

// Twiddle table: tw4[j*32 + l] = (W^{l*2j}, W^{l*(2j+1)}), W = exp(+i 2 pi / 1024),
// filled by `nthreads` threads with indices `tid`.
__device__ __forceinline__ void wfft_twiddles(float4* tw4, int tid, int nthreads) {
    for (int idx = tid; idx < WShape::TW4; idx += nthreads) {
        const int j = idx >> 5, l = idx & 31;
        float s0, c0, s1, c1;
        sincospif((float)((l * 2 * j) & 1023) / 512.0f, &s0, &c0);
        sincospif((float)((l * (2 * j + 1)) & 1023) / 512.0f, &s1, &c1);
        tw4[idx] = make_float4(c0, s0, c1, s1);
    }
}

// v[c] of lane l is element (l, c) of a 32 x 32 matrix; on return v[r] of
// lane l is element (r, l).  xb: this warp's XBUF float2 of shared memory.
// Rows are written as 16-byte pairs (a row stride of 17 float4 spreads the 8
// lanes of each quarter-warp over distinct banks) and read as columns (one
// float2 per lane, consecutive).  Ends with the buffer free for reuse.
__device__ __forceinline__ void wfft_transpose(float2* v, float2* xb, int l) {
    float4* xb4 = reinterpret_cast<float4*>(xb);
#pragma unroll
    for (int j = 0; j < 16; ++j)
        xb4[l * (WShape::XS / 2) + j] = make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x,
                                                    v[2 * j + 1].y);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = xb[r * WShape::XS + l];
    __syncwarp();
}

// Forward transform of the warp's 1024 points: p = l + 32 i in, k = l + 32 i
// out (see the file comment).
__device__ __forceinline__ void wfft_forward(float2* v, float2* xb, const float4* tw4, int l) {
    dft32<-1>(v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float4 t = tw4[j * 32 + l];
        if (j) v[2 * j] = cmulc(v[2 * j], make_float2(t.x, t.y));
        v[2 * j + 1] = cmulc(v[2 * j + 1], make_float2(t.z, t.w));
    }
    wfft_transpose(v, xb, l);
    dft32<-1>(v);
}

// Inverse transform of the warp's 1024 frequencies (k = l + 32 i), without
// 1/L: p = l + 32 i out.  The two passes run as one rolled
// loop so that the 32-point DFT is compiled once.
__device__ __forceinline__ void wfft_inverse(float2* v, float2* xb, const float4* tw4, int l) {
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        dft32<1>(v);
        if (pass == 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 t = tw4[j * 32 + l];
                if (j) v[2 * j] = cmul_p(v[2 * j], make_float2(t.x, t.y));
                v[2 * j + 1] = cmul_p(v[2 * j + 1], make_float2(t.z, t.w));
            }
            wfft_transpose(v, xb, l);
        }
    }
}

}  // namespace fdas
