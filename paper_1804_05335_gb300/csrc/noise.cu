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
// One CTA per plane row evaluates, one per thread, the 2h + 1 responses at
// integer offsets (kept in shared memory for the half-bin differences) and
// the 2h at half-integer ones, in FP64 (R from fresnel.cuh), then reduces the
// three sums across its warps.
#include "fresnel.cuh"
#include "internal.h"

namespace fdas {

constexpr int kNoiseThreads = 512;

__global__ void __launch_bounds__(kNoiseThreads) noise_means_kernel(int zmin, int zstep, int K,
                                                                    int interbin,
                                                                    float* __restrict__ out) {
    extern __shared__ double2 rs[];   // Rt(d) at rs[d + h + 1], d = -h-1 .. h+1
    __shared__ double part[3][kNoiseThreads / 32];
    const int row = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int z = zmin + row * zstep;
    const int az = z < 0 ? -z : z;
    const int h = (az + 1) / 2 + 8;
    const int nint = 2 * h + 1;
    double e_full = 0.0, e_half = 0.0, e_mid = 0.0;
    for (int i = threadIdx.x; i < nint + 2 * h; i += kNoiseThreads) {
        if (i < nint) {   // integer offset d = i - h
            const cd r = response<double>((double)z, (double)(i - h));
            rs[i + 1] = make_double2(r.x, r.y);
            e_full += r.x * r.x + r.y * r.y;
        } else {          // half-integer offset d - 1/2, d = -h+1 .. h
            const cd r = response<double>((double)z, (double)(i - nint - h + 1) - 0.5);
            e_mid += r.x * r.x + r.y * r.y;
        }
    }
    if (threadIdx.x == 0) rs[0] = make_double2(0.0, 0.0);           // Rt(-h-1)
    if (threadIdx.x == 1) rs[2 * h + 2] = make_double2(0.0, 0.0);   // Rt(h+1)
    __syncthreads();
    for (int d = -h + (int)threadIdx.x; d <= h + 1; d += kNoiseThreads) {
        const double2 a = rs[d + h + 1], b = rs[d + h];   // Rt(d), Rt(d - 1)
        const double dx = a.x - b.x, dy = a.y - b.y;
        e_half += dx * dx + dy * dy;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        e_full += __shfl_xor_sync(0xffffffffu, e_full, o);
        e_half += __shfl_xor_sync(0xffffffffu, e_half, o);
        e_mid += __shfl_xor_sync(0xffffffffu, e_mid, o);
    }
    if (lane == 0) {
        part[0][warp] = e_full;
        part[1][warp] = e_half;
        part[2][warp] = e_mid;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        e_full = e_half = e_mid = 0.0;
        for (int w = 0; w < kNoiseThreads / 32; ++w) {
            e_full += part[0][w];
            e_half += part[1][w];
            e_mid += part[2][w];
        }
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
    const size_t sm = (size_t)(2 * g.hmax + 3) * sizeof(double2);   // <= 32.8 KB (h <= 1023)
    noise_means_kernel<<<g.K, kNoiseThreads, sm, (cudaStream_t)stream>>>(p->zmin, p->zstep, g.K,
                                                                           p->interbin, means);
    return cuda_status(cudaGetLastError());
}
