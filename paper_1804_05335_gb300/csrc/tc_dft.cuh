// The L = 1024 convolver's 32-point DFT passes on the tensor cores (tcgen05),
// the split-precision form of Section 4.2's DFT as a matrix product
// (Eq. matrixDFT) for the warp layout of wfft.cuh.
//
// In one pass every lane of the CTA's 4 warps holds one DFT instance (its 32
// complex values), so the 128 lanes are the 128 rows of
//   D (128 x 64, FP32, tensor memory) = A (128 x 64) x W (64 x 64),
// with x as the real row [x0.re, x0.im, x1.re, ...] and W the real form of the
// inverse DFT, W[2j][2m] = W[2j+1][2m+1] = Re w^{jm}, W[2j+1][2m] = -Im w^{jm},
// W[2j][2m+1] = Im w^{jm}, w = exp(+i 2 pi / 32).  Both operands are split
// into 16-bit parts, x = x_hi + x_lo (+ x_mid), W likewise, and the products
// kept are those of order up to 2^-16 of the leading one:
//   PREC 1 (FP16 hi+lo):     Xh Wh + Xh Wl + Xl Wh, each instance scaled by a
//                            power of two into FP16's range first;
//   PREC 2 (BF16 hi+lo):     the same three products, unscaled;
//   PREC 3 (BF16 hi+mid+lo): Xh Wh + Xh Wm + Xm Wh + Xh Wl + Xl Wh + Xm Wm.
// The forward transform is the inverse of the conjugated input, conjugated.
//
// A lives in tensor memory (each lane writes its row, two 16-bit values per
// 32-bit column: real part low, imaginary high), W in shared memory in the
// no-swizzle K-major layout (8 x 8 cores of 16-byte rows; cores 128 B apart
// along K, 1024 B apart along N), D in tensor memory read back one row per
// lane.  One thread issues the 4 K-steps of every product and commits them
// to an mbarrier; the hand-offs use mbarriers with bounded waits (no CTA
// barrier that a stopped warp could leave waiting): each warp's lane 0
// arrives on `ready` once its rows are stored, the issuing thread waits for
// all four, and every thread waits on `done` before reading D.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tma.cuh"

namespace fdas {

template <int PREC>
struct TcShape {
    static constexpr int PARTS = PREC == 3 ? 3 : 2;
    static constexpr int DCOL = 32 * PARTS;                    // D columns DCOL .. DCOL + 63
    static constexpr int NCOLS = DCOL + 64 <= 128 ? 128 : 256; // tensor memory allocated
    static constexpr int BPART = 64 * 64 * 2;                   // bytes of one W part
    static constexpr int BBYTES = PARTS * BPART;
};

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    // start >> 4 | leading (K) byte offset 128 >> 4 | stride (N) byte offset
    // 1024 >> 4 | descriptor version 1 | base offset 0 | no swizzle
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 D; A and B both F16 (fmt 0) or BF16
// (fmt 1); K-major A and B; N = 64, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(int fmt) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(64 >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ uint32_t tc_pack(float a, float b) {
    if constexpr (PREC == 1) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <int PREC>
__device__ __forceinline__ float2 tc_unpack(uint32_t u) {
    if constexpr (PREC == 1) return __half22float2(*reinterpret_cast<__half2*>(&u));
    else return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&u));
}

// The W parts into shared memory (all threads of the CTA, nthreads of them).
// Element (k, n) of part q sits at byte q*BPART + ((n/8)*8 + k/8)*128 +
// (n%8)*16 + (k%8)*2.
template <int PREC>
__device__ void tc_fill_w(unsigned char* wsm, int tid, int nthreads) {
    for (int idx = tid; idx < 64 * 64; idx += nthreads) {
        const int k = idx & 63, n = idx >> 6;
        const int j = k >> 1, m = n >> 1;
        float s, c;
        sincospif((float)((j * m) & 31) / 16.0f, &s, &c);   // w^{jm}, w = exp(+i 2 pi/32)
        const int ck = k & 1, cn = n & 1;
        const float val = ck == cn ? c : (ck ? -s : s);
        const int off = ((n >> 3) * 8 + (k >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
        float rem = val;
        for (int q = 0; q < TcShape<PREC>::PARTS; ++q) {
            uint16_t h;
            if constexpr (PREC == 1) {
                const __half x = __float2half_rn(rem);
                h = *reinterpret_cast<const uint16_t*>(&x);
                rem -= __half2float(x);
            } else {
                const __nv_bfloat16 x = __float2bfloat16_rn(rem);
                h = *reinterpret_cast<const uint16_t*>(&x);
                rem -= __bfloat162float(x);
            }
            *reinterpret_cast<uint16_t*>(wsm + q * TcShape<PREC>::BPART + off) = h;
        }
    }
}

__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
          "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]),
          "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]),
          "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
          "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* f) {
    uint32_t* r = reinterpret_cast<uint32_t*>(f);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc,
                                       uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d), "r"(a), "l"(bdesc), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
        ::"r"(smem_u32(bar)) : "memory");
}

// Per-CTA state of the tensor-core passes.
struct TcCtx {
    uint32_t tmem;     // base address of the CTA's tensor memory
    uint32_t wsm;      // shared address of the W parts
    uint64_t* ready;   // 4 arrivals (one per warp): rows stored
    uint64_t* done;    // 1 arrival (commit): products finished
    uint32_t phase;    // passes completed so far (parity of both barriers)
    uint32_t commits;  // issuing thread: passes whose products it committed
};

// One 32-point inverse DFT of v (32 complex) per lane, on the tensor cores.
// Every thread of the CTA calls it the same number of times.  Returns false
// if a bounded wait ran out (abort is then set); v is then undefined.
template <int PREC>
__device__ __forceinline__ bool tc_dft32(float2* v, TcCtx& c, int tid, volatile int* abort,
                                         uint32_t limit) {
    using TS = TcShape<PREC>;
    const int w = tid >> 5, l = tid & 31;
    const uint32_t row = c.tmem + ((uint32_t)(32 * w) << 16);
    float si = 1.f, so = 1.f;
    if constexpr (PREC == 1) {
        // power-of-two scale bringing the largest component into [2^14, 2^15)
        uint32_t mb = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            mb = max(mb, max(__float_as_uint(v[j].x) & 0x7fffffffu, __float_as_uint(v[j].y) & 0x7fffffffu));
        const int e = (int)(mb >> 23);
        const int k = min(max(141 - e, -100), 100);
        si = __uint_as_float((uint32_t)(127 + k) << 23);
        so = __uint_as_float((uint32_t)(127 - k) << 23);
    }
    uint32_t p[32];
#pragma unroll
    for (int q = 0; q < TS::PARTS; ++q) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float a = q == 0 ? v[j].x * si : v[j].x, b = q == 0 ? v[j].y * si : v[j].y;
            p[j] = tc_pack<PREC>(a, b);
            const float2 h = tc_unpack<PREC>(p[j]);
            v[j] = make_float2(a - h.x, b - h.y);   // remainder for the next part
        }
        tc_st32(row + 32u * q, p);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncwarp();
    if (l == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(c.ready)) : "memory");
    const uint32_t par = c.phase & 1u;
    bool ok = true;
    if (tid == 0) {
        ok = mbar_wait_bounded(c.ready, par, limit) && !*abort;
        if (ok) {
            tc_fence_after();
            constexpr uint32_t idesc = tc_idesc(PREC == 1 ? 0 : 1);
            const uint32_t d = c.tmem + TS::DCOL;
            // (A part, W part) pairs, smallest first; part 0 = hi, then (mid,) lo
            constexpr int NPROD = PREC == 3 ? 6 : 3;
            constexpr int pa3[6] = {0, 2, 1, 0, 1, 0}, pb3[6] = {2, 0, 1, 1, 0, 0};
            constexpr int pa2[3] = {1, 0, 0}, pb2[3] = {0, 1, 0};
#pragma unroll
            for (int pr = 0; pr < NPROD; ++pr) {
                const int ia = PREC == 3 ? pa3[pr] : pa2[pr];
                const int ib = PREC == 3 ? pb3[pr] : pb2[pr];
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    tc_mma(d, c.tmem + 32u * ia + 8u * ks,
                           tc_desc(c.wsm + ib * TS::BPART + ks * 256), idesc,
                           (pr | ks) ? 1u : 0u);
            }
            tc_commit(c.done);
            c.commits = c.phase + 1;
        }
    }
    ok = (tid == 0 ? ok : true) && mbar_wait_bounded(c.done, par, limit);
    ++c.phase;
    if (!__all_sync(0xffffffffu, ok)) {
        if (l == 0) *abort = 1;
        return false;
    }
    tc_fence_after();
    float* f = reinterpret_cast<float*>(v);
    tc_ld32(row + TS::DCOL, f);
    tc_ld32(row + TS::DCOL + 32, f + 32);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if constexpr (PREC == 1) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = make_float2(v[j].x * so, v[j].y * so);
    }
    return true;
}

}  // namespace fdas
