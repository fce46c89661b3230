// fdas_make_templates: FP64 template responses (Fresnel integrals) and their
// L-point spectra, stored FP32 in the convolver's digit-reversed order.  The
// spectra come from the convolver's own forward FFT, so no reordering is
// ever needed (Section 4.2: the templates must be transformed by the same
// algorithm as the segments).
//
// The response R_z(d) and its FP64 / FP32 evaluation are described in
// fresnel.cuh.
#include <math.h>

#include "conv_fft.cuh"
#include "fresnel.cuh"
#include "internal.h"

namespace fdas {

constexpr int kTapThreads = 128;

// Kernel 1: one thread per (bank row b, tap j), |j| <= sub*h.  Writes the
// FIR kernel taps g[j] = conj(R_z(-j/sub)) / L (sub = 1: one tap per bin;
// sub = 2: half-bin sampling for 2-bin Fourier interpolation, the template
// at twice the resolution) to the start of bank row b as tap index
// j + sub*h (float2), where the row-b CTA of kernel 2 reads them before it
// overwrites the row.
__global__ void __launch_bounds__(kTapThreads) template_taps_kernel(int L, int zfirst, int zstep,
                                                                    int width, int rows, int sub,
                                                                    float2* __restrict__ bank) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= rows * width) return;
    const int b = gid / width, idx = gid - b * width;
    const int z = zfirst + b * zstep;
    const int az = z < 0 ? -z : z;
    const int hh = sub * ((az + 1) / 2 + 8);
    if (idx > 2 * hh) return;
    const int j = idx - hh;                      // tap position (circular index j mod L)
    const cd r = response<float>((double)z, -(double)j / (double)sub);
    const double s = 1.0 / (double)L;
    bank[(size_t)b * (L + 16) + idx] = make_float2((float)(r.x * s), (float)(-r.y * s));
}

// Kernel 2: one CTA of L/16 threads per bank row: gather the circularly
// placed kernel g (D1 distribution), forward FFT with the convolver's own
// permutation-free transform, store the digit-reversed spectrum in place.
template <int L>
__global__ void __launch_bounds__(L / 16) template_fft_kernel(int zfirst, int zstep, int sub,
                                                              float2* __restrict__ bank) {
    using S = ConvShape<L>;
    constexpr int T = S::T;
    extern __shared__ float4 tsm4[];
    float2* buf0 = reinterpret_cast<float2*>(tsm4);
    float2* buf1 = buf0 + S::BUFS;
    const int b = blockIdx.x, t = threadIdx.x;
    const int z = zfirst + b * zstep;
    const int az = z < 0 ? -z : z;
    const int h = sub * ((az + 1) / 2 + 8);
    float2* row = bank + (size_t)b * S::ROW;
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int p = i * T + t;
        const int j = p <= h ? p : p - L;        // circular tap position
        v[i] = (j >= -h && j <= h) ? row[j + h] : make_float2(0.f, 0.f);
    }
    __syncthreads();   // every tap is read before the row is overwritten
    forward_fft_d3<L>(v, buf0, buf1, t);
    float4* row4 = reinterpret_cast<float4*>(row);
#pragma unroll
    for (int ip = 0; ip < 8; ++ip)
        row4[ip * T + t] = make_float4(v[2 * ip].x, v[2 * ip].y, v[2 * ip + 1].x, v[2 * ip + 1].y);
    if (t == 0) {
        // mirror slots: float4 L/2 + j holds (H[-k(2ip+1)], H[-k(2ip)]) of thread 0, ip = 7 - j,
        // so that the conjugate-template read of thread 0 has the same form as everyone's
        constexpr int Q = S::Q;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int ip = 7 - j;
            const float2 hi = v[thread0_mirror<Q>(2 * ip + 1)], lo = v[thread0_mirror<Q>(2 * ip)];
            row4[L / 2 + j] = make_float4(hi.x, hi.y, lo.x, lo.y);
        }
    }
}

template <int L>
static int launch_fft(int rows, int zfirst, int zstep, int sub, float2* bank, cudaStream_t st) {
    constexpr size_t sm = 2 * ConvShape<L>::BUFS * sizeof(float2);
    const int rc = kernel_setup(reinterpret_cast<const void*>(&template_fft_kernel<L>), sm, L / 16,
                                nullptr, nullptr);
    if (rc != FDAS_OK) return rc;
    template_fft_kernel<L><<<rows, L / 16, sm, st>>>(zfirst, zstep, sub, bank);
    return cuda_status(cudaGetLastError());
}

int launch_templates(const fdas_params* p, const Grid& g, float2* bank, cudaStream_t st) {
    const int sub = p->interbin == 2 ? 2 : 1;   // taps per bin
    const int width = 2 * sub * g.hmax + 1;
    if (width > p->L + 16) return FDAS_E_UNSUPPORTED;
    const int zfirst = p->zmin + g.j0 * p->zstep;
    const int total = g.Kb * width;
    template_taps_kernel<<<(total + kTapThreads - 1) / kTapThreads, kTapThreads, 0, st>>>(
        p->L, zfirst, p->zstep, width, g.Kb, sub, bank);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return FDAS_E_CUDA;
    switch (p->L) {
        case 1024: return launch_fft<1024>(g.Kb, zfirst, p->zstep, sub, bank, st);
        case 2048: return launch_fft<2048>(g.Kb, zfirst, p->zstep, sub, bank, st);
        case 4096: return launch_fft<4096>(g.Kb, zfirst, p->zstep, sub, bank, st);
        default: return FDAS_E_INVAL;
    }
}

}  // namespace fdas
