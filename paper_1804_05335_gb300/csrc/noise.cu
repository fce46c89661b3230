// fdas_noise_means: mean noise power of every plane row, for significance
// (the paper leaves the statistics of single-bin, interbinned and Fourier-
// interpolated powers open, Section 5.2).
//
// After normalisation the spectrum is unit-variance complex Gaussian noise,
// A_k ~ CN(0, 1) independent, so a plane value is |G|^2 for a complex
// Gaussian G and is exponential with mean E|G|^2:
//   full bin      F_r = sum_{|d|<=h} A_{r+d} conj(R(d)):    sum_{|d|<=h} |R(d)|^2
//   half bin      (pi/4)(F_r - F_{r+1}):    (pi/4)^2 sum_d |Rt(d) - Rt(d-1)|^2,
//                 Rt = R on |d| <= h and 0 outside
//   half-integer  F(r + 1/2) (2-bin interpolation):    sum_{|d|<=h, d in Z+1/2} |R(d)|^2
// One warp per plane row sums over the taps in FP64 (R from fresnel.cuh).
#include "fresnel.cuh"
#include "internal.h"

namespace fdas {

__global__ void noise_means_kernel(int zmin, int zstep, int K, int interbin, float* __restrict__ out) {
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= K) return;
    const int z = zmin + row * zstep;
    const int az = z < 0 ? -z : z;
    const int h = (az + 1) / 2 + 8;
    double e_full = 0.0, e_half = 0.0, e_mid = 0.0;
    for (int d = -h + lane; d <= h + 1; d += 32) {
        // Rt(d) and Rt(d - 1) (zero outside the window), R(d - 1/2)
        const cd r0 = (d <= h) ? response<double>((double)z, (double)d) : cd{0.0, 0.0};
        const cd r1 = (d - 1 >= -h) ? response<double>((double)z, (double)(d - 1)) : cd{0.0, 0.0};
        if (d <= h) e_full += r0.x * r0.x + r0.y * r0.y;
        const double dx = r0.x - r1.x, dy = r0.y - r1.y;
        e_half += dx * dx + dy * dy;
        if (d <= h) {   // half-integer offset d - 1/2 inside the window: |d - 1/2| <= h - 1/2
            if (d - 1 >= -h) {
                const cd rm = response<double>((double)z, (double)d - 0.5);
                e_mid += rm.x * rm.x + rm.y * rm.y;
            }
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        e_full += __shfl_xor_sync(0xffffffffu, e_full, o);
        e_half += __shfl_xor_sync(0xffffffffu, e_half, o);
        e_mid += __shfl_xor_sync(0xffffffffu, e_mid, o);
    }
    if (lane == 0) {
        const double hs = 0.61685027506808491;   // (pi/4)^2
        out[2 * row] = (float)e_full;
        out[2 * row + 1] = (float)(interbin == 1 ? hs * e_half : interbin == 2 ? e_mid : e_full);
    }
}

}  // namespace fdas

using namespace fdas;

extern "C" int fdas_noise_means(const fdas_params* p, float* means, void* stream) {
    Grid g;
    int rc = make_grid(p, &g);
    if (rc != FDAS_OK) return rc;
    if (!means || !aligned(means, 4)) return FDAS_E_INVAL;
    constexpr int kWarps = 4;
    noise_means_kernel<<<(g.K + kWarps - 1) / kWarps, 32 * kWarps, 0, (cudaStream_t)stream>>>(
        p->zmin, p->zstep, g.K, p->interbin, means);
    return cuda_status(cudaGetLastError());
}
