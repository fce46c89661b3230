// fdas_correlate_plane16: the FP32 convolver writing its plane as 16-bit
// floats (kernel in conv_kernel.cuh, element type OUT = 1 half, 2 bfloat16).
// Single-series launches only.
#include "conv_kernel.cuh"

namespace fdas {

template <int OUT>
static int dispatch_plane16(const fdas_params* p, const ConvArgs& a, bool fused, cudaStream_t st) {
    switch (p->L) {
        case 1024:
            return dispatch_wconv(p, a, fused, false, OUT, 0, st);
        case 2048:
            return fused ? launch_one<2048, true, false, 0, OUT>(a, 0, st)
                         : launch_one<2048, false, false, 0, OUT>(a, 0, st);
        case 4096:
            return fused ? launch_one<4096, true, false, 0, OUT>(a, 0, st)
                         : launch_one<4096, false, false, 0, OUT>(a, 0, st);
        default:
            return FDAS_E_INVAL;
    }
}

int launch_correlate_plane16(const fdas_params* p, const Grid& g, int type, const float2* spec,
                             int64_t nb, const float4* bank, void* plane, int64_t row_stride,
                             const fdas_fused_threshold* fused, int32_t* status, cudaStream_t st) {
    ConvArgs a = base_args(p, g, bank, fused, status);
    a.spec = spec;
    a.nb = nb;
    a.plane = static_cast<float*>(plane);   // addressed as 16-bit elements by the kernel
    a.row_stride = row_stride;
    a.items = series_items(g, p->L, positions(p, nb));
    if (fused) {
        cudaError_t e = cudaMemsetAsync(fused->count, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) return FDAS_E_CUDA;
    }
    switch (type) {
        case FDAS_PLANE_F16: return dispatch_plane16<1>(p, a, fused != nullptr, st);
        case FDAS_PLANE_BF16: return dispatch_plane16<2>(p, a, fused != nullptr, st);
        default: return FDAS_E_INVAL;
    }
}

}  // namespace fdas
