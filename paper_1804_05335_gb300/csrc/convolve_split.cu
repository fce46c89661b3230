// fdas_correlate_split: the convolver with its radix-16 DFT passes as
// split-precision tensor-core products: warp-level mma.sync in the CTA
// convolver for L = 2048 and 4096 (conv_kernel.cuh, split_mma.cuh), tcgen05
// with tensor memory in the warp convolver for L = 1024 (wconv_split.cu,
// tc_dft.cuh).  Single-series launches.
#include "conv_kernel.cuh"

namespace fdas {

template <int PREC>
static int dispatch_split(const fdas_params* p, const ConvArgs& a, bool fused, cudaStream_t st) {
    switch (p->L) {
        case 1024:
            return dispatch_wconv_split(p, a, fused, PREC, st);
        case 2048:
            return fused ? launch_one<2048, true, false, PREC>(a, 0, st)
                         : launch_one<2048, false, false, PREC>(a, 0, st);
        case 4096:
            return fused ? launch_one<4096, true, false, PREC>(a, 0, st)
                         : launch_one<4096, false, false, PREC>(a, 0, st);
        default:
            return FDAS_E_INVAL;
    }
}

int launch_correlate_split(const fdas_params* p, const Grid& g, int prec, const float2* spec,
                           int64_t nb, const float4* bank, float* plane, int64_t row_stride,
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
    switch (prec) {
        case FDAS_PREC_FP16_SPLIT: return dispatch_split<1>(p, a, fused != nullptr, st);
        case FDAS_PREC_BF16_SPLIT: return dispatch_split<2>(p, a, fused != nullptr, st);
        case FDAS_PREC_BF16_SPLIT3: return dispatch_split<3>(p, a, fused != nullptr, st);
        default: return FDAS_E_INVAL;
    }
}

}  // namespace fdas
