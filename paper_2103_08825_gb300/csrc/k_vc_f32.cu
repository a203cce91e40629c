// k_vc_f32.cu -- the variable-coefficient kernels for STENCIL_F32 storage.
#include "k_vc.cuh"

namespace sg {
cudaError_t launch_vc_F32(const stencil_plan_s &P, int k, const void *coef, const void *src, void *dst,
                         cudaStream_t st) {
    return launch_vc_dt<STENCIL_F32>(P, k, coef, src, dst, st);
}
}  // namespace sg
