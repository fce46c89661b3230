// fdas_correlate and fdas_correlate_batched: launchers of the FP32 convolver
// (kernel in conv_kernel.cuh; L = 1024 goes to the warp convolver, wconv.cu).
#include "conv_kernel.cuh"

namespace fdas {

template <bool BATCH>
static int dispatch(const fdas_params* p, const ConvArgs& a, bool fused, int ctas_per_sm,
                    cudaStream_t st) {
    if (p->L == 1024) return dispatch_wconv(p, a, fused, BATCH, 0, ctas_per_sm, st);
    if (p->interbin == 2) return dispatch_half_bins(p, a, fused, BATCH, ctas_per_sm, st);
    switch (p->L) {
        case 2048:
            return fused ? launch_one<2048, true, BATCH>(a, ctas_per_sm, st)
                         : launch_one<2048, false, BATCH>(a, ctas_per_sm, st);
        case 4096:
            return fused ? launch_one<4096, true, BATCH>(a, ctas_per_sm, st)
                         : launch_one<4096, false, BATCH>(a, ctas_per_sm, st);
        default:
            return FDAS_E_INVAL;
    }
}

int launch_correlate(const fdas_params* p, const Grid& g, const float2* spec, int64_t nb,
                     const float4* bank, float* plane, int64_t row_stride,
                     const fdas_fused_threshold* fused, int32_t* status, cudaStream_t st) {
    ConvArgs a = base_args(p, g, bank, fused, status);
    a.spec = spec;
    a.nb = nb;
    a.plane = plane;
    a.row_stride = row_stride;
    a.items = series_items(g, p->L, positions(p, nb));
    if (fused) {
        cudaError_t e = cudaMemsetAsync(fused->count, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return FDAS_E_CUDA;
    }
    return dispatch<false>(p, a, fused != nullptr, 0, st);
}

int launch_correlate_batched(const fdas_params* p, const Grid& g, const fdas_trial* trials,
                             int32_t ntrials, int64_t total_items, const float4* bank,
                             const fdas_fused_threshold* fused, int ctas_per_sm, int tpb,
                             int32_t* status, cudaStream_t st) {
    ConvArgs a = base_args(p, g, bank, fused, status);
    a.tpb = tpb;
    a.trials = trials;
    a.ntrials = ntrials;
    a.items = total_items;
    if (fused) {
        cudaError_t e = cudaMemsetAsync(fused->count, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return FDAS_E_CUDA;
    }
    return dispatch<true>(p, a, fused != nullptr, ctas_per_sm, st);
}

}  // namespace fdas
