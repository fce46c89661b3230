// fdas_threshold: candidates of a power plane (Section 3: the power is
// compared with a pre-computed threshold), with an optional local-maximum
// flag over the 8 neighbours.
#include "internal.h"

namespace fdas {

constexpr int kThrThreads = 256;

__device__ __forceinline__ bool is_peak(const float* __restrict__ plane, int rows, int64_t width,
                                        int64_t stride, int row, int64_t col, float v) {
#pragma unroll
    for (int dr = -1; dr <= 1; ++dr) {
#pragma unroll
        for (int dc = -1; dc <= 1; ++dc) {
            if (dr == 0 && dc == 0) continue;
            const int rr = row + dr;
            const int64_t cc = col + dc;
            if (rr < 0 || rr >= rows || cc < 0 || cc >= width) continue;
            const float w = __ldg(&plane[(int64_t)rr * stride + cc]);
            const bool before = (dr < 0) || (dr == 0 && dc < 0);
            if (before ? !(v > w) : !(v >= w)) return false;
        }
    }
    return true;
}

// Each thread takes kThrVec groups of 4 columns, kThrThreads groups apart, and
// loads all of them before comparing (enough bytes in flight per SM to keep
// the plane read streaming).
constexpr int kThrVec = 4;

__global__ void __launch_bounds__(kThrThreads) threshold_kernel(
    const float* __restrict__ plane, int rows, int64_t width, int64_t stride, float thr,
    int want_peak, fdas_cand* __restrict__ out, int cap, int* __restrict__ count,
    int* __restrict__ status, int vec) {
    const int row = blockIdx.y;
    const float* prow = plane + (int64_t)row * stride;
    float v[kThrVec][4];
#pragma unroll
    for (int g = 0; g < kThrVec; ++g) {
        const int64_t c0 = (((int64_t)blockIdx.x * kThrVec + g) * kThrThreads + threadIdx.x) * 4;
        if (vec && c0 + 3 < width) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(prow + c0));
            v[g][0] = q.x; v[g][1] = q.y; v[g][2] = q.z; v[g][3] = q.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[g][e] = (c0 + e < width) ? __ldg(prow + c0 + e) : thr;
        }
    }
#pragma unroll
    for (int g = 0; g < kThrVec; ++g) {
        const int64_t c0 = (((int64_t)blockIdx.x * kThrVec + g) * kThrThreads + threadIdx.x) * 4;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (v[g][e] > thr) {
                const int64_t col = c0 + e;
                int flags = 0;
                if (want_peak && is_peak(plane, rows, width, stride, row, col, v[g][e]))
                    flags = FDAS_CAND_PEAK;
                const int idx = atomicAdd(count, 1);
                if (idx < cap) {
                    fdas_cand c;
                    c.z_idx = row;
                    c.col = (int32_t)col;
                    c.power = v[g][e];
                    c.flags = flags;
                    out[idx] = c;
                } else if (status) {
                    atomicOr(status, FDAS_STATUS_OVERFLOW);
                }
            }
        }
    }
}

}  // namespace fdas

using namespace fdas;

extern "C" int fdas_threshold(const float* plane, int32_t rows, int64_t width, int64_t row_stride,
                              float thr, int32_t want_flags, fdas_cand* out, int32_t cap,
                              int32_t* count, int32_t* status, void* stream) {
    if (!plane || !count || rows < 1 || rows > 65535 || width < 1 || row_stride < width ||
        cap < 0 || (cap > 0 && !out) || width > ((int64_t)1 << 31))
        return FDAS_E_INVAL;
    if (!aligned(plane, 4) || !aligned(count, 4) || (status && !aligned(status, 4)))
        return FDAS_E_INVAL;
    if (want_flags & ~FDAS_CAND_PEAK) return FDAS_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess) return FDAS_E_CUDA;
    const int vec = (aligned(plane, 16) && (row_stride % 4) == 0) ? 1 : 0;
    const int64_t per_cta = (int64_t)4 * kThrThreads * kThrVec;
    dim3 grid((unsigned)((width + per_cta - 1) / per_cta), (unsigned)rows);
    threshold_kernel<<<grid, kThrThreads, 0, st>>>(plane, rows, width, row_stride, thr,
                                                    want_flags & FDAS_CAND_PEAK, out, cap, count,
                                                    status, vec);
    return cuda_status(cudaGetLastError());
}
