// fdas_make_templates: FP64 template responses (Fresnel integrals) and their
// L-point spectra, stored FP32 in the order the convolver for L reads them
// (digit-reversed for the CTA convolver of L = 2048, 4096; natural order in
// the warp layout for L = 1024).  The spectra come from the convolver's own
// forward FFT (Section 4.2: the templates must be transformed by the same
// algorithm as the segments).
//
// The response R_z(d) and its FP64 / FP32 evaluation are described in
// fresnel.cuh.
#include <math.h>

#include "conv_fft.cuh"
#include "fresnel.cuh"
#include "internal.h"
#include "wfft.cuh"

namespace fdas {

constexpr int kTapThreads = 128;

// Kernel 1: one thread per (bank row b, tap j), |j| <= sub*h.  Writes the
// FIR kernel taps g[j] = conj(R_z(-j/sub)) / L (sub = 1: one tap per bin;
// sub = 2: half-bin sampling for 2-bin Fourier interpolation, the template
// at twice the resolution) to the start of bank row b as tap index
// j + sub*h (float2; rows of rowc complex values), where kernel 2 reads them
// before it overwrites the row.
__global__ void __launch_bounds__(kTapThreads) template_taps_kernel(int L, int rowc, int zfirst,
                                                                    int zstep, int width, int rows,
                                                                    int sub, float2* __restrict__ bank) {
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
    bank[(size_t)b * rowc + idx] = make_float2((float)(r.x * s), (float)(-r.y * s));
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

// Kernel 2 for L = 1024: one warp per bank row.  Gathers the circularly placed
// kernel (position p = l + 32 i in lane l, register i), runs the convolver's
// warp FFT (wfft.cuh) and stores H[k], k = l + 32 i, as float4 slot
// j*33 + l = (H[l + 64 j], H[l + 64 j + 32]); lane 0 also fills the mirror
// column, slot j*33 + 32 = (H[64 j + 32], H[(64 j + 64) mod 1024]), which holds
// the values lane 0 needs for a conjugated (-z) template.
constexpr int kWRowsPerCta = 4;
__global__ void __launch_bounds__(kWRowsPerCta * 32) wtemplate_fft_kernel(int rows, int zfirst,
                                                                          int zstep, int sub,
                                                                          float4* __restrict__ bank) {
    extern __shared__ float4 wts4[];
    float4* tw4 = wts4;
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    float2* xb = reinterpret_cast<float2*>(wts4 + WShape::TW4) + w * WShape::XBUF;
    wfft_twiddles(tw4, tid, kWRowsPerCta * 32);
    __syncthreads();
    const int b = blockIdx.x * kWRowsPerCta + w;
    if (b >= rows) return;
    const int z = zfirst + b * zstep;
    const int az = z < 0 ? -z : z;
    const int h = sub * ((az + 1) / 2 + 8);
    float4* row4 = bank + (size_t)b * WShape::ROW4;
    const float2* taps = reinterpret_cast<const float2*>(row4);
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int p = l + 32 * i;
        const int j = p <= h ? p : p - WShape::L;   // circular tap position
        v[i] = (j >= -h && j <= h) ? taps[j + h] : make_float2(0.f, 0.f);
    }
    __syncwarp();   // every tap is read before the row is overwritten
    wfft_forward(v, xb, tw4, l);
#pragma unroll
    for (int j = 0; j < 16; ++j)
        row4[j * 33 + l] = make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
    if (l == 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            row4[j * 33 + 32] = make_float4(v[2 * j + 1].x, v[2 * j + 1].y, v[(2 * j + 2) & 31].x,
                                            v[(2 * j + 2) & 31].y);
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
    if (width > bank_row_complex(p->L)) return FDAS_E_UNSUPPORTED;
    const int zfirst = p->zmin + g.j0 * p->zstep;
    const int total = g.Kb * width;
    template_taps_kernel<<<(total + kTapThreads - 1) / kTapThreads, kTapThreads, 0, st>>>(
        p->L, bank_row_complex(p->L), zfirst, p->zstep, width, g.Kb, sub, bank);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return FDAS_E_CUDA;
    switch (p->L) {
        case 1024: {
            constexpr size_t sm = (size_t)WShape::TW4 * sizeof(float4) +
                                  (size_t)kWRowsPerCta * WShape::XBUF * sizeof(float2);
            const int rc = kernel_setup(reinterpret_cast<const void*>(&wtemplate_fft_kernel), sm,
                                        kWRowsPerCta * 32, nullptr, nullptr);
            if (rc != FDAS_OK) return rc;
            wtemplate_fft_kernel<<<(g.Kb + kWRowsPerCta - 1) / kWRowsPerCta, kWRowsPerCta * 32, sm,
                                   st>>>(g.Kb, zfirst, p->zstep, sub,
                                         reinterpret_cast<float4*>(bank));
            return cuda_status(cudaGetLastError());
        }
        case 2048: return launch_fft<2048>(g.Kb, zfirst, p->zstep, sub, bank, st);
        case 4096: return launch_fft<4096>(g.Kb, zfirst, p->zstep, sub, bank, st);
        default: return FDAS_E_INVAL;
    }
}

}  // namespace fdas
