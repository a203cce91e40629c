// k_fused3d_f32.cu -- the 3D fused kernel for STENCIL_F32 storage, radius 1,
// and its dispatcher (radii 2 and 3: k_fused3d_f32_r23.cu; one translation
// unit each keeps the build parallel).
#include "k_fused3d.cuh"

namespace sg {
extern template cudaError_t launch_f3_r<STENCIL_F32, 2>(const stencil_plan_s &, const void *, void *, int,
                                                         cudaStream_t);
extern template cudaError_t launch_f3_r<STENCIL_F32, 3>(const stencil_plan_s &, const void *, void *, int,
                                                         cudaStream_t);
cudaError_t launch_f3_F32(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f3_dt<STENCIL_F32>(P, src, dst, k, st);
}
cudaError_t launch_f3_all_F32(const stencil_plan_s &P, const void *src, void *const *lv, int k, cudaStream_t st) {
    if (P.dim != 3 || P.r != 1 || P.dtype != STENCIL_F32 || fused3d_max_k(P) < 1) return cudaErrorNotSupported;
    return P.pattern == STENCIL_BOX ? launch_f3_all_k<STENCIL_F32, STENCIL_BOX>(P, src, lv, k, st)
                                    : launch_f3_all_k<STENCIL_F32, STENCIL_STAR>(P, src, lv, k, st);
}
}  // namespace sg
