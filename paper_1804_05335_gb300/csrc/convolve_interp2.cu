// The FP32 convolver with half-bin sampling (interbin = 2, 2-bin Fourier
// interpolation): conv_kernel with SUB = 2, single-series and batched.
#include "conv_kernel.cuh"

namespace fdas {

template <bool BATCH>
static int dispatch_sub2(const fdas_params* p, const ConvArgs& a, bool fused, int ctas_per_sm,
                         cudaStream_t st) {
    switch (p->L) {
        case 2048:
            return fused ? launch_one<2048, true, BATCH, 0, 0, 2>(a, ctas_per_sm, st)
                         : launch_one<2048, false, BATCH, 0, 0, 2>(a, ctas_per_sm, st);
        case 4096:
            return fused ? launch_one<4096, true, BATCH, 0, 0, 2>(a, ctas_per_sm, st)
                         : launch_one<4096, false, BATCH, 0, 0, 2>(a, ctas_per_sm, st);
        default:
            return FDAS_E_INVAL;
    }
}

int dispatch_half_bins(const fdas_params* p, const ConvArgs& a, bool fused, bool batch,
                       int ctas_per_sm, cudaStream_t st) {
    return batch ? dispatch_sub2<true>(p, a, fused, ctas_per_sm, st)
                 : dispatch_sub2<false>(p, a, fused, ctas_per_sm, st);
}

}  // namespace fdas
