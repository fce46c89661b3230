// fdas_correlate_split for L = 1024: the warp convolver with its 32-point DFT
// passes on the tensor cores (tcgen05, tc_dft.cuh).  Single-series launches.
#include "wconv_kernel.cuh"

namespace fdas {

template <int PREC>
static int launch_prec(const ConvArgs& a, bool fused, bool ib, cudaStream_t st) {
    if (ib)
        return fused ? launch_w<true, false, 0, 1, true, PREC>(a, 0, st)
                     : launch_w<false, false, 0, 1, true, PREC>(a, 0, st);
    return fused ? launch_w<true, false, 0, 1, false, PREC>(a, 0, st)
                 : launch_w<false, false, 0, 1, false, PREC>(a, 0, st);
}

int dispatch_wconv_split(const fdas_params* p, const ConvArgs& a, bool fused, int prec,
                         cudaStream_t st) {
    if (p->interbin == 2) return FDAS_E_UNSUPPORTED;
    const bool ib = p->interbin == 1;
    switch (prec) {
        case FDAS_PREC_FP16_SPLIT: return launch_prec<1>(a, fused, ib, st);
        case FDAS_PREC_BF16_SPLIT: return launch_prec<2>(a, fused, ib, st);
        case FDAS_PREC_BF16_SPLIT3: return launch_prec<3>(a, fused, ib, st);
        default: return FDAS_E_INVAL;
    }
}

}  // namespace fdas
