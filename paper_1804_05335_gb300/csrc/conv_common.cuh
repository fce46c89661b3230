// Pieces shared by the two overlap-save convolver kernels (Sections 3, 4.1,
// 4.2): the launch arguments, the work-item bookkeeping of template groups and
// of +-z pairs, candidate emission, the plane stores for every element type,
// and the per-series state of batched launches.
//   conv_kernel.cuh   L = 2048, 4096: one CTA per segment FFT (16 x 16 x L/256)
//   wconv_kernel.cuh  L = 1024: one warp per segment FFT (32 x 32)
#pragma once
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dft.cuh"
#include "internal.h"

namespace fdas {

struct ConvArgs {
    const float2* spec;
    int64_t nb;
    const float4* bank;
    float* plane;
    int64_t row_stride;
    int64_t items;      // nseg * K
    int32_t K;
    int32_t j0;
    int32_t sym;
    int32_t zero;
    int32_t M;
    int32_t interbin;
    float thr;
    fdas_cand* cand;
    int32_t cap;
    int32_t* count;
    int32_t* status;
    const fdas_trial* trials;   // batched launches: device table of ntrials series
    int32_t ntrials;
    // template groups (Grid): overlap, first bank row and template count of
    // each; a series' items are group-major, segment-major within a group
    int32_t ng;
    uint32_t wait_limit;   // polls of a bounded wait before it gives up (0: kWaitLimit)
    int32_t probe;         // diagnostic (L = 1024): arm the first row's barrier, issue no copy
    int32_t tpb;           // L = 1024: templates per chunk of a group's unit order (0: all)
    int32_t gM[kMaxGroups];
    int32_t gb0[kMaxGroups];
    int32_t gK[kMaxGroups];
};

// polls of a template-row bulk copy before a kernel gives up
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ void emit(const ConvArgs& A, int row, int64_t col, float v, int flags) {
    int idx = atomicAdd(A.count, 1);
    if (idx < A.cap) {
        fdas_cand c;
        c.z_idx = row;
        c.col = (int32_t)col;
        c.power = v;
        c.flags = flags;
        A.cand[idx] = c;
    } else if (A.status) {
        atomicOr(A.status, FDAS_STATUS_OVERFLOW);
    }
}

// Template q of group g inside a segment: bank row, plane row, conjugation.
// Items of a symmetric grid pair +z with -z so that both use one bank row;
// group g holds bank rows gb0[g] onwards (z = 0 first in group 0).
__device__ __forceinline__ void item_row(const ConvArgs& A, int g, int q, int& row, int& brow,
                                         int& cj) {
    if (!A.sym) {
        row = q; brow = q; cj = 0;
        return;
    }
    const int b0 = A.gb0[g];
    if (A.zero && b0 == 0) {
        if (q == 0) { brow = 0; cj = 0; }
        else { brow = (q + 1) >> 1; cj = (q & 1) ? 0 : 1; }
    } else {
        brow = b0 + (q >> 1); cj = q & 1;
    }
    row = cj ? (A.K - 1 - A.j0 - brow) : (A.j0 + brow);
}

// Segments of a series of nb bins in group g.
__device__ __forceinline__ int64_t group_segments(const ConvArgs& A, int L, int g, int64_t nb) {
    const int64_t B = L - A.gM[g];
    return (nb + B - 1) / B;
}

// Plane stores by element type OUT (0 float, 1 IEEE half, 2 bfloat16; values
// rounded to nearest): 4, 2 or 1 consecutive elements from element i of a row.
// The 4- and 2-element stores are streaming and need 4-element alignment
// (16 bytes for float, 8 for the 16-bit types) and 2-element alignment.
template <int OUT>
__device__ __forceinline__ void plane_store4(void* row, int64_t i, float4 v) {
    if constexpr (OUT == 0) {
        __stcs(reinterpret_cast<float4*>(static_cast<float*>(row) + i), v);
    } else {
        uint2 u;
        if constexpr (OUT == 1) {
            __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
            u = make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
        } else {
            __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
            u = make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
        }
        __stcs(reinterpret_cast<uint2*>(static_cast<uint16_t*>(row) + i), u);
    }
}
template <int OUT>
__device__ __forceinline__ void plane_store2(void* row, int64_t i, float2 v) {
    if constexpr (OUT == 0) {
        __stcs(reinterpret_cast<float2*>(static_cast<float*>(row) + i), v);
    } else {
        uint32_t u;
        if constexpr (OUT == 1) {
            __half2 a = __floats2half2_rn(v.x, v.y);
            u = *reinterpret_cast<uint32_t*>(&a);
        } else {
            __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
            u = *reinterpret_cast<uint32_t*>(&a);
        }
        __stcs(reinterpret_cast<unsigned int*>(static_cast<uint16_t*>(row) + i), u);
    }
}
template <int OUT>
__device__ __forceinline__ void plane_store1(void* row, int64_t i, float v) {
    if constexpr (OUT == 0) {
        static_cast<float*>(row)[i] = v;
    } else if constexpr (OUT == 1) {
        reinterpret_cast<__half*>(row)[i] = __float2half_rn(v);
    } else {
        reinterpret_cast<__nv_bfloat16*>(row)[i] = __float2bfloat16_rn(v);
    }
}

// Powers of one pair of positions (j, j+1) given x[j], x[j+1], x[j+2].
__device__ __forceinline__ float4 pair_powers(float4 x01, float2 xn) {
    const float hs = 0.61685027506808491f;   // (pi/4)^2
    const float2 x0 = make_float2(x01.x, x01.y), x1 = make_float2(x01.z, x01.w);
    const float2 d0 = x0 - x1, d1 = x1 - xn;
    return make_float4(fmaf(x0.x, x0.x, x0.y * x0.y), hs * fmaf(d0.x, d0.x, d0.y * d0.y),
                       fmaf(x1.x, x1.x, x1.y * x1.y), hs * fmaf(d1.x, d1.x, d1.y * d1.y));
}

// Series state of the item being processed: one series for fdas_correlate,
// the trial table entry for fdas_correlate_batched.
struct SeriesState {
    const float2* spec;
    int64_t nb;
    float* plane;
    int64_t row_stride;
    int64_t end;   // first item of the next series
    int flags;     // candidate flags: trial index << 8 in batched launches
};

template <bool BATCH>
__device__ __forceinline__ SeriesState series_of(const ConvArgs& A, int trial) {
    SeriesState st;
    if constexpr (BATCH) {
        const fdas_trial& tr = A.trials[trial];
        st.spec = reinterpret_cast<const float2*>(tr.spec);
        st.nb = tr.nb;
        st.plane = tr.plane;
        st.row_stride = tr.row_stride;
        st.end = (trial + 1 < A.ntrials) ? A.trials[trial + 1].item_begin : A.items;
        st.flags = trial << 8;
    } else {
        st.spec = A.spec;
        st.nb = A.nb;
        st.plane = A.plane;
        st.row_stride = A.row_stride;
        st.end = A.items;
        st.flags = 0;
    }
    return st;
}

// Launch arguments common to every entry point.
inline ConvArgs base_args(const fdas_params* p, const Grid& g, const float4* bank,
                          const fdas_fused_threshold* fused, int32_t* status) {
    ConvArgs a;
    a.spec = nullptr;
    a.nb = 0;
    a.plane = nullptr;
    a.row_stride = 0;
    a.items = 0;
    a.bank = bank;
    a.K = g.K;
    a.ng = g.ng;
    for (int k = 0; k < kMaxGroups; ++k) {
        a.gM[k] = k < g.ng ? g.gM[k] : p->M;
        a.gb0[k] = k < g.ng ? g.gb0[k] : 0;
        a.gK[k] = k < g.ng ? g.gK[k] : 1;
    }
    a.j0 = g.j0;
    a.sym = g.sym;
    a.zero = g.zero;
    a.M = p->M;
    a.interbin = p->interbin;
    a.thr = fused ? fused->thr : 0.f;
    a.cand = fused ? fused->out : nullptr;
    a.cap = fused ? fused->cap : 0;
    a.count = fused ? fused->count : nullptr;
    a.status = status;
    a.trials = nullptr;
    a.ntrials = 0;
    a.wait_limit = 0;
    a.probe = 0;
    a.tpb = 0;
    return a;
}

}  // namespace fdas
