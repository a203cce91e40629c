// k_fused2d_mp_f16.cu -- instantiations of the persistent multi-pass 2D kernel for
// STENCIL_F16 storage, radius 1, and its dispatcher (radius 2: k_fused2d_mp_f16_r2.cu).
#include "k_fused2d.cuh"

namespace sg {
extern template cudaError_t launch_f2mp_r<STENCIL_F16, 2>(const stencil_plan_s &, const void *, void *, void *, int,
                                                            int, cudaStream_t);
cudaError_t launch_f2mp_F16(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                            cudaStream_t st) {
    return launch_f2mp_dt<STENCIL_F16>(P, src0, de, dof, k, passes, st);
}
}  // namespace sg
