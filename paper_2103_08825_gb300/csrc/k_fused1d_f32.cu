// k_fused1d_f32.cu -- the 1D fused kernels (one launch per pass and
// persistent multi-pass) for STENCIL_F32 storage, radii 1..3, depths 1..16.
#include "k_fused1d.cuh"

namespace sg {
cudaError_t launch_f1_F32(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f1_dt<STENCIL_F32>(P, src, dst, k, st);
}
cudaError_t launch_f1mp_F32(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                            cudaStream_t st) {
    return launch_f1mp_dt<STENCIL_F32>(P, src0, de, dof, k, passes, st);
}
}  // namespace sg
