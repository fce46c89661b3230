// fdas_harmonic_sum: incremental harmonic summing on the f-fdot plane with a
// fused threshold (the search stage after the plane that the paper names as
// the next to move on chip, Sections 3 and 7).
//
// A periodic signal with fundamental (r, z) has its h-th harmonic at (h r,
// h z).  On the plane, row j holds z_j = zmin + j zstep and column c holds
// r = c/2 (interbinned) or r = c, so harmonic h of (j, c) sits at column h c
// and at row j_h = (h - 1) zmin / zstep + h j, which is a grid row whenever
// zmin is a multiple of zstep.  For every fundamental whose second harmonic
// is on the plane a thread forms
//   S_2 = P[j][c] + P[j_2][2c],  S_4 = S_2 + P[j_3][3c] + P[j_4][4c],
//   S_8 = S_4 + P[j_5][5c] + ... + P[j_8][8c],
// stopping at the first level whose harmonics leave the plane, and lists
// (row j, column c, S_H, H) for every S_H above that level's threshold.
// A block takes 1024 consecutive fundamentals of one row, four per thread.
// fdas_harmonic_sum launches the blocks row by row; fdas_harmonic_sum_planned
// takes them from a plan sorted by u = c / |z/zstep|, the quantity a
// fundamental shares with all its harmonics, so that the rows reading the
// same plane sectors run together and L2 serves the repeats.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "internal.h"

namespace fdas {

constexpr int kHarmThreads = 256;
constexpr int kHarmPer = 4;   // fundamentals per thread

template <int TYPE>
__device__ __forceinline__ float plane_load(const void* plane, int64_t i) {
    if constexpr (TYPE == 0) {
        return __ldg(static_cast<const float*>(plane) + i);
    } else if constexpr (TYPE == 1) {
        return __half2float(__ldg(static_cast<const __half*>(plane) + i));
    } else {
        return __bfloat162float(__ldg(static_cast<const __nv_bfloat16*>(plane) + i));
    }
}

struct HarmArgs {
    const void* plane;
    int64_t width, row_stride;
    int32_t K, j0h;          // plane rows; j0h = zmin / zstep (row offset of harmonic rows)
    int32_t nlev;            // levels: 1 -> H = 2, 2 -> up to 4, 3 -> up to 8
    float thr[3];
    fdas_cand* out;
    int32_t cap;
    int32_t* count;
    int32_t* status;
};

__device__ __forceinline__ void harm_emit(const HarmArgs& A, int row, int64_t col, float v, int H) {
    const int idx = atomicAdd(A.count, 1);
    if (idx < A.cap) {
        fdas_cand c;
        c.z_idx = row;
        c.col = (int32_t)col;
        c.power = v;
        c.flags = H;
        A.out[idx] = c;
    } else if (A.status) {
        atomicOr(A.status, FDAS_STATUS_OVERFLOW);
    }
}

// Sums and thresholds of a thread's fundamentals from their loaded
// harmonics (nl[f] levels on the plane for fundamental f).
__device__ __forceinline__ void harm_sums(const HarmArgs& A, int j, int64_t c0,
                                          const float (&v)[kHarmPer][8], const int (&nl)[kHarmPer]) {
#pragma unroll
    for (int f = 0; f < kHarmPer; ++f) {
        if (nl[f] == 0) continue;
        const int64_t c = c0 + f * kHarmThreads;
        float s = v[f][0] + v[f][1];
        if (s > A.thr[0]) harm_emit(A, j, c, s, 2);
        if (nl[f] < 2) continue;
        s += v[f][2] + v[f][3];
        if (s > A.thr[1]) harm_emit(A, j, c, s, 4);
        if (nl[f] < 3) continue;
        s += (v[f][4] + v[f][5]) + (v[f][6] + v[f][7]);
        if (s > A.thr[2]) harm_emit(A, j, c, s, 8);
    }
}

// A thread whose fundamentals all have NL levels on the plane: harmonic h of
// fundamental f is element h (ra + c0) - rb + h f 256 (the row offsets are
// linear in h, ra and rb as in harm_block), so each harmonic takes one
// address and kHarmPer loads at fixed offsets from it.
template <int TYPE, int NL>
__device__ __forceinline__ void harm_block_full(const HarmArgs& A, int j, int64_t c0,
                                                int64_t ra, int64_t rb) {
    constexpr int H = 2 << (NL - 1);
    float v[kHarmPer][8];
    int nl[kHarmPer];
#pragma unroll
    for (int h = 1; h <= 8; ++h) {
#pragma unroll
        for (int f = 0; f < kHarmPer; ++f) {
            v[f][h - 1] = 0.f;
            if (h <= H) v[f][h - 1] = plane_load<TYPE>(A.plane, h * (ra + c0) - rb +
                                                                    h * f * kHarmThreads);
        }
    }
#pragma unroll
    for (int f = 0; f < kHarmPer; ++f) nl[f] = NL;
    harm_sums(A, j, c0, v, nl);
}

// One CTA: fundamentals c = blk * kHarmBlock + threadIdx.x + f * kHarmThreads
// (f < kHarmPer) of fundamental row j.  Each thread issues every load of all
// its fundamentals before forming the sums.  Harmonic rows j_h = h (j + j0h)
// - j0h are linear in h, so the harmonics up to H are all on the plane when
// j_H is; the levels whose columns are on the plane fall as c grows, so the
// thread's fundamentals share their level count unless its first and last
// differ.
constexpr int kHarmBlock = kHarmThreads * kHarmPer;

template <int TYPE>
__device__ __forceinline__ void harm_block(const HarmArgs& A, int j, int64_t blk) {
    int nlr = 0;   // levels whose harmonic rows are on the plane
    for (int lev = 0; lev < A.nlev; ++lev) {
        const int H = 2 << lev;
        const int jH = (H - 1) * A.j0h + H * j;
        if (jH < 0 || jH >= A.K) break;
        nlr = lev + 1;
    }
    // harmonic h's row starts at ((h - 1) j0h + h j) row_stride = h ra - rb
    const int64_t ra = (int64_t)(A.j0h + j) * A.row_stride, rb = (int64_t)A.j0h * A.row_stride;
    const int64_t c0 = blk * kHarmBlock + threadIdx.x;
    auto levels = [&](int64_t c) {
        int n = 0;   // levels whose columns are on the plane too
        while (n < nlr && ((int64_t)2 << n) * c < A.width) ++n;
        return n;
    };
    const int nfirst = levels(c0), nlast = levels(c0 + (kHarmPer - 1) * kHarmThreads);
    if (nfirst == nlast) {   // the same levels for all of the thread's fundamentals
        if (nlast == 3) harm_block_full<TYPE, 3>(A, j, c0, ra, rb);
        else if (nlast == 2) harm_block_full<TYPE, 2>(A, j, c0, ra, rb);
        else if (nlast == 1) harm_block_full<TYPE, 1>(A, j, c0, ra, rb);
        return;
    }
    // a level boundary falls between them: per-fundamental levels
    float v[kHarmPer][8];
    int nl[kHarmPer];
#pragma unroll
    for (int f = 0; f < kHarmPer; ++f) {
        const int64_t c = c0 + f * kHarmThreads;
        const int n = levels(c);
        nl[f] = n;
#pragma unroll
        for (int h = 1; h <= 8; ++h) {
            const int need = h <= 2 ? 1 : (h <= 4 ? 2 : 3);
            v[f][h - 1] = 0.f;
            if (need <= n) v[f][h - 1] = plane_load<TYPE>(A.plane, h * (ra + c) - rb);
        }
    }
    harm_sums(A, j, c0, v, nl);
}

// Row-major order: x over groups of kRowPer column blocks, y over the
// fundamental rows.
constexpr int kRowPer = 16;

template <int TYPE>
// 6 CTAs per SM (at most 42 registers, a few bytes spilled): the kernels are held by
// memory latency, and more warps keep more loads in flight (measured: 4 CTAs
// 0.98 ms, 5 CTAs 0.81 ms, 6 CTAs 0.80 ms, 8 CTAs 0.87 ms planned on the FP32
// production plane)
__global__ void __launch_bounds__(kHarmThreads, 6) harmonic_kernel(const HarmArgs A, int jlo,
                                                                int64_t nblk) {
    for (int g = 0; g < kRowPer; ++g) {
        const int64_t blk = (int64_t)blockIdx.x * kRowPer + g;
        if (blk >= nblk) break;
        harm_block<TYPE>(A, jlo + (int)blockIdx.y, blk);
    }
}

// Ray-ordered launch: block b takes entry b of a plan, (row j, column block).
// The plan header holds what it was made for; a mismatch lists nothing.
constexpr int32_t kPlanMagic = 0x48504c31;   // "HPL1"
constexpr int kPlanHeaderWords = 16;         // int32 words before the entries (64 bytes)
constexpr int kPlanPer = 8;                  // plan entries per block

template <int TYPE>
__global__ void __launch_bounds__(kHarmThreads, 6) harmonic_planned_kernel(const HarmArgs A,
                                                                       const int32_t* hdr) {
    const int64_t width = (int64_t)(uint32_t)hdr[3] | ((int64_t)hdr[4] << 32);
    if (hdr[0] != kPlanMagic || hdr[1] != A.K || hdr[2] != A.j0h || width != A.width) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && A.status)
            atomicOr(A.status, FDAS_STATUS_BADPLAN);
        return;
    }
    const int2* ent = reinterpret_cast<const int2*>(hdr + kPlanHeaderWords);
    const int n = hdr[5];
    for (int g = 0; g < kPlanPer; ++g) {
        const int i = blockIdx.x * kPlanPer + g;
        if (i >= n) break;
        const int2 e = ent[i];
        harm_block<TYPE>(A, e.x, (int64_t)e.y);
    }
}

// Fundamental rows (second harmonic on the plane) and column blocks of a
// plan; false for invalid arguments or more than 2^31 - 1 blocks.
static bool plan_shape(const fdas_params* p, int64_t width, Grid* g, int* jlo, int* jhi,
                       int64_t* nblk) {
    if (make_grid(p, g) != FDAS_OK || p->zmin % p->zstep != 0 || width < 1 || width > INT32_MAX)
        return false;
    const int j0h = p->zmin / p->zstep;
    *jlo = 0;
    *jhi = -1;
    for (int j = 0; j < g->K; ++j) {
        const int j2 = j0h + 2 * j;
        if (j2 >= 0 && j2 < g->K) {
            if (*jhi < 0) *jlo = j;
            *jhi = j;
        }
    }
    const int64_t nc = (width + 1) / 2;
    *nblk = (nc + kHarmBlock - 1) / kHarmBlock;
    const int64_t rows = *jhi >= *jlo ? *jhi - *jlo + 1 : 0;
    return rows * *nblk < ((int64_t)1 << 31);
}

}  // namespace fdas

using namespace fdas;

extern "C" size_t fdas_harmonic_plan_bytes(const fdas_params* p, int64_t width) {
    Grid g;
    int jlo, jhi;
    int64_t nblk;
    if (!plan_shape(p, width, &g, &jlo, &jhi, &nblk)) return 0;
    const int64_t n = (jhi >= jlo ? jhi - jlo + 1 : 0) * nblk;
    return (size_t)(4 * kPlanHeaderWords + 8 * n + 15) / 16 * 16;
}

extern "C" int fdas_harmonic_plan(const fdas_params* p, int64_t width, void* plan,
                                  size_t plan_bytes) {
    Grid g;
    int jlo, jhi;
    int64_t nblk;
    if (!plan_shape(p, width, &g, &jlo, &jhi, &nblk)) return FDAS_E_INVAL;
    if (!plan || !aligned(plan, 16) || plan_bytes < fdas_harmonic_plan_bytes(p, width))
        return FDAS_E_INVAL;
    const int j0h = p->zmin / p->zstep;
    const int64_t rows = jhi >= jlo ? jhi - jlo + 1 : 0;
    std::vector<std::pair<double, int64_t>> key((size_t)(rows * nblk));
    size_t i = 0;
    for (int j = jlo; j <= jhi; ++j) {
        const int ay = std::abs(j + j0h);
        for (int64_t b = 0; b < nblk; ++b, ++i) {
            // u of the block's middle; the z = 0 row (no u) first, in column order
            const double u = ay ? (b + 0.5) / ay : -1.0 + (double)b / (double)nblk;
            key[i] = {u, (int64_t)j * nblk + b};
        }
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<double, int64_t>& x, const std::pair<double, int64_t>& y) {
                         return x.first < y.first;
                     });
    std::vector<int32_t> host((size_t)(kPlanHeaderWords + 2 * key.size()), 0);
    host[0] = kPlanMagic;
    host[1] = g.K;
    host[2] = j0h;
    host[3] = (int32_t)(uint32_t)(width & 0xffffffff);
    host[4] = (int32_t)(width >> 32);
    host[5] = (int32_t)key.size();
    for (size_t e = 0; e < key.size(); ++e) {
        host[kPlanHeaderWords + 2 * e] = (int32_t)(key[e].second / nblk);
        host[kPlanHeaderWords + 2 * e + 1] = (int32_t)(key[e].second % nblk);
    }
    return cuda_status(cudaMemcpy(plan, host.data(), host.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice));
}

namespace fdas {

// Checks shared by both harmonic-sum entries; fills the kernel arguments and
// the range of fundamental rows [jlo, jhi] (jhi < jlo: none).
static int harmonic_args(const fdas_params* p, int32_t plane_type, const void* plane,
                         int64_t width, int64_t row_stride, int32_t nlevels, const float* thr,
                         fdas_cand* out, int32_t cap, int32_t* count, int32_t* status,
                         HarmArgs* a, int* jlo, int* jhi) {
    Grid g;
    int rc = make_grid(p, &g);
    if (rc != FDAS_OK) return rc;
    if (plane_type < 0 || plane_type > 2 || !plane || !thr || !out || !count) return FDAS_E_INVAL;
    if (nlevels < 1 || nlevels > 3 || width < 1 || width > INT32_MAX || row_stride < width ||
        cap < 0)
        return FDAS_E_INVAL;
    if (p->zmin % p->zstep != 0) return FDAS_E_INVAL;   // harmonic rows must be grid rows
    if (!aligned(plane, plane_type == 0 ? 4 : 2) || !aligned(out, 4) || !aligned(count, 4))
        return FDAS_E_INVAL;
    if (status && !aligned(status, 4)) return FDAS_E_INVAL;
    a->plane = plane;
    a->width = width;
    a->row_stride = row_stride;
    a->K = g.K;
    a->j0h = p->zmin / p->zstep;
    a->nlev = nlevels;
    for (int l = 0; l < 3; ++l) a->thr[l] = l < nlevels ? thr[l] : 0.f;
    a->out = out;
    a->cap = cap;
    a->count = count;
    a->status = status;
    // fundamental rows whose second harmonic row 2 j + j0h lies in [0, K)
    *jlo = 0;
    *jhi = -1;
    for (int j = 0; j < g.K; ++j) {
        const int j2 = a->j0h + 2 * j;
        if (j2 >= 0 && j2 < g.K) {
            if (*jhi < 0) *jlo = j;
            *jhi = j;
        }
    }
    return FDAS_OK;
}

}  // namespace fdas

extern "C" int fdas_harmonic_sum(const fdas_params* p, int32_t plane_type, const void* plane,
                                 int64_t width, int64_t row_stride, int32_t nlevels,
                                 const float* thr, fdas_cand* out, int32_t cap, int32_t* count,
                                 int32_t* status, void* stream) {
    HarmArgs a;
    int jlo, jhi;
    const int rc = harmonic_args(p, plane_type, plane, width, row_stride, nlevels, thr, out, cap,
                                 count, status, &a, &jlo, &jhi);
    if (rc != FDAS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess) return FDAS_E_CUDA;
    if (jhi < 0) return FDAS_OK;
    const int64_t nc = (width + 1) / 2;
    const int64_t nblk = (nc + kHarmBlock - 1) / kHarmBlock;
    const dim3 grid((unsigned)((nblk + kRowPer - 1) / kRowPer), (unsigned)(jhi - jlo + 1));
    switch (plane_type) {
        case 0: harmonic_kernel<0><<<grid, kHarmThreads, 0, st>>>(a, jlo, nblk); break;
        case 1: harmonic_kernel<1><<<grid, kHarmThreads, 0, st>>>(a, jlo, nblk); break;
        default: harmonic_kernel<2><<<grid, kHarmThreads, 0, st>>>(a, jlo, nblk); break;
    }
    return cuda_status(cudaGetLastError());
}

extern "C" int fdas_harmonic_sum_planned(const fdas_params* p, int32_t plane_type,
                                         const void* plane, int64_t width, int64_t row_stride,
                                         int32_t nlevels, const float* thr, fdas_cand* out,
                                         int32_t cap, int32_t* count, int32_t* status,
                                         const void* plan, size_t plan_bytes, void* stream) {
    HarmArgs a;
    int jlo, jhi;
    const int rc = harmonic_args(p, plane_type, plane, width, row_stride, nlevels, thr, out, cap,
                                 count, status, &a, &jlo, &jhi);
    if (rc != FDAS_OK) return rc;
    const size_t need = fdas_harmonic_plan_bytes(p, width);
    if (need == 0 || !plan || !aligned(plan, 16) || plan_bytes < need) return FDAS_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess) return FDAS_E_CUDA;
    if (jhi < 0) return FDAS_OK;
    const int64_t nc = (width + 1) / 2;
    const int64_t n = (int64_t)(jhi - jlo + 1) * ((nc + kHarmBlock - 1) / kHarmBlock);
    const int32_t* hdr = static_cast<const int32_t*>(plan);
    const int64_t nb = (n + kPlanPer - 1) / kPlanPer;
    switch (plane_type) {
        case 0: harmonic_planned_kernel<0><<<(unsigned)nb, kHarmThreads, 0, st>>>(a, hdr); break;
        case 1: harmonic_planned_kernel<1><<<(unsigned)nb, kHarmThreads, 0, st>>>(a, hdr); break;
        default: harmonic_planned_kernel<2><<<(unsigned)nb, kHarmThreads, 0, st>>>(a, hdr); break;
    }
    return cuda_status(cudaGetLastError());
}
