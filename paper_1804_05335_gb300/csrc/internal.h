// Library-internal declarations shared by the FDAS translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fdas.h"

namespace fdas {

constexpr int kMaxGroups = FDAS_MAX_GROUPS;
// L = 1024 convolver: warps per CTA, each holding one of a unit's segments
constexpr int kWarpSegments = 4;
// ... and its CTAs per SM (registers allow 168 per thread)
constexpr int kWarpCtasPerSm = 12 / kWarpSegments;

// Template grid and bank-row bookkeeping derived from fdas_params.
struct Grid {
    int32_t K;       // templates (plane rows)
    int32_t Kb;      // bank rows
    int32_t j0;      // number of z < 0 rows served by conjugation (symmetric grid), else 0
    int32_t sym;     // 1: symmetric grid, bank holds z >= 0 only
    int32_t zero;    // 1: z = 0 is on a symmetric grid
    int32_t hmax;    // largest half-width on the grid
    // Template groups of increasing |z| (symmetric grids; one group otherwise),
    // each convolved with the smallest overlap its longest template needs.
    int32_t ng;
    int32_t gM[kMaxGroups];    // overlap (discarded points per segment) of group g
    int32_t gb0[kMaxGroups];   // first bank row of group g
    int32_t gK[kMaxGroups];    // templates (plane rows) of group g
};

// Validates p; returns FDAS_OK and fills g (groups included), or FDAS_E_INVAL.
int make_grid(const fdas_params* p, Grid* g);

// Positions of the correlation for nb spectral bins: nb, or 2 nb with
// half-bin (2-bin Fourier interpolation) sampling.
inline int64_t positions(const fdas_params* p, int64_t nb) { return p->interbin == 2 ? 2 * nb : nb; }

// Work items of one series of npos positions.  L = 2048, 4096 (one CTA per
// segment FFT): (segment, template) pairs, for each group ceil(npos / (L - gM))
// segments times gK templates.  L = 1024 (one warp per segment FFT): units of
// one template on kWarpSegments consecutive segments, ceil(segments /
// kWarpSegments) times gK.
int64_t series_items(const Grid& g, int L, int64_t npos);

// Complex values per template-bank row: L = 1024 rows hold 16 register pairs
// x 33 slots (32 lanes + a mirror column) of two values; longer segments hold
// L digit-reversed values + 16 mirror slots.
inline int bank_row_complex(int L) { return L == 1024 ? L + 32 : L + 16; }

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? FDAS_OK : FDAS_E_CUDA; }

inline bool aligned(const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// Once per (kernel, current device), thread-safe: allow `smem` bytes of
// dynamic shared memory for kernel `fn`, and report the device's SM count and
// how many CTAs of `threads` threads with that shared memory fit on one SM.
// FDAS_OK, FDAS_E_CUDA, or FDAS_E_UNSUPPORTED when not even one CTA fits.
// carveout >= 0: also the preferred shared-memory carveout (percent), set once
int kernel_setup(const void* fn, size_t smem, int threads, int* sms, int* per_sm,
                 int carveout = -1);

// Launchers implemented in the .cu files.
int launch_templates(const fdas_params* p, const Grid& g, float2* bank, cudaStream_t st);
int launch_correlate(const fdas_params* p, const Grid& g, const float2* spec, int64_t nb,
                     const float4* bank, float* plane, int64_t row_stride,
                     const fdas_fused_threshold* fused, int32_t* status, cudaStream_t st);
int launch_correlate_batched(const fdas_params* p, const Grid& g, const fdas_trial* trials,
                             int32_t ntrials, int64_t total_items, const float4* bank,
                             const fdas_fused_threshold* fused, int ctas_per_sm, int tpb,
                             int32_t* status, cudaStream_t st);
struct ConvArgs;
// The L = 1024 (one warp per segment FFT) convolver, wconv.cu: element type
// `out` (0 float, FDAS_PLANE_F16, FDAS_PLANE_BF16), half-bin sampling when
// p->interbin == 2.
int dispatch_wconv(const fdas_params* p, const ConvArgs& a, bool fused, bool batch, int out,
                   int ctas_per_sm, cudaStream_t st);
// The L = 1024 convolver with its DFT passes on the tensor cores
// (fdas_correlate_split, wconv_split.cu).
int dispatch_wconv_split(const fdas_params* p, const ConvArgs& a, bool fused, int prec,
                         cudaStream_t st);
// The L = 1024 convolver with its first template row's barrier armed and
// no copy issued, `polls` polls per wait (fdas_debug_wait_timeout).
int launch_wconv_wait_probe(const fdas_params* p, const Grid& g, const float2* spec, int64_t nb,
                            const float4* bank, float* plane, int64_t row_stride, uint32_t polls,
                            int32_t* status, cudaStream_t st);
// The convolver with half-bin sampling (interbin 2), convolve_interp2.cu.
int dispatch_half_bins(const fdas_params* p, const ConvArgs& a, bool fused, bool batch,
                       int ctas_per_sm, cudaStream_t st);
int launch_correlate_plane16(const fdas_params* p, const Grid& g, int type, const float2* spec,
                             int64_t nb, const float4* bank, void* plane, int64_t row_stride,
                             const fdas_fused_threshold* fused, int32_t* status, cudaStream_t st);
int launch_correlate_split(const fdas_params* p, const Grid& g, int prec, const float2* spec,
                           int64_t nb, const float4* bank, float* plane, int64_t row_stride,
                           const fdas_fused_threshold* fused, int32_t* status, cudaStream_t st);

}  // namespace fdas
