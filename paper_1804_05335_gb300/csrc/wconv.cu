// Launchers of the L = 1024 convolver (one warp per segment FFT, kernel in
// wconv_kernel.cuh) for fdas_correlate, fdas_correlate_batched,
// fdas_correlate_plane16 and 2-bin Fourier interpolation (interbin 2).
#include "wconv_kernel.cuh"

namespace fdas {

template <bool BATCH, int OUT, int SUB>
static int launch_fused(const ConvArgs& a, bool fused, int interbin, int ctas_per_sm,
                        cudaStream_t st) {
    if constexpr (SUB == 1) {
        if (interbin == 1)
            return fused ? launch_w<true, BATCH, OUT, SUB, true>(a, ctas_per_sm, st)
                         : launch_w<false, BATCH, OUT, SUB, true>(a, ctas_per_sm, st);
    }
    return fused ? launch_w<true, BATCH, OUT, SUB, false>(a, ctas_per_sm, st)
                 : launch_w<false, BATCH, OUT, SUB, false>(a, ctas_per_sm, st);
}

int dispatch_wconv(const fdas_params* p, const ConvArgs& a, bool fused, bool batch, int out,
                   int ctas_per_sm, cudaStream_t st) {
    if (p->interbin == 2) {
        if (out != 0) return FDAS_E_UNSUPPORTED;
        return batch ? launch_fused<true, 0, 2>(a, fused, p->interbin, ctas_per_sm, st)
                     : launch_fused<false, 0, 2>(a, fused, p->interbin, ctas_per_sm, st);
    }
    switch (out) {
        case 0:
            return batch ? launch_fused<true, 0, 1>(a, fused, p->interbin, ctas_per_sm, st)
                         : launch_fused<false, 0, 1>(a, fused, p->interbin, ctas_per_sm, st);
        case FDAS_PLANE_F16:
            if (batch) return FDAS_E_UNSUPPORTED;
            return launch_fused<false, 1, 1>(a, fused, p->interbin, ctas_per_sm, st);
        case FDAS_PLANE_BF16:
            if (batch) return FDAS_E_UNSUPPORTED;
            return launch_fused<false, 2, 1>(a, fused, p->interbin, ctas_per_sm, st);
        default:
            return FDAS_E_INVAL;
    }
}

int launch_wconv_wait_probe(const fdas_params* p, const Grid& g, const float2* spec, int64_t nb,
                            const float4* bank, float* plane, int64_t row_stride, uint32_t polls,
                            int32_t* status, cudaStream_t st) {
    ConvArgs a = base_args(p, g, bank, nullptr, status);
    a.spec = spec;
    a.nb = nb;
    a.plane = plane;
    a.row_stride = row_stride;
    a.items = series_items(g, p->L, positions(p, nb));
    a.wait_limit = polls;
    a.probe = 1;
    return dispatch_wconv(p, a, false, false, 0, 0, st);
}

}  // namespace fdas
