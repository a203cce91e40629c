// k_fused2d_mp_f64.cu -- instantiations of the persistent multi-pass 2D kernel for
// STENCIL_F64 storage, radius 1, and its dispatcher (radius 2: k_fused2d_mp_f64_r2.cu).
#include "k_fused2d.cuh"

namespace sg {
extern template cudaError_t launch_f2mp_r<STENCIL_F64, 2>(const stencil_plan_s &, const void *, void *, void *, int,
                                                            int, cudaStream_t);
cudaError_t launch_f2mp_F64(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                            cudaStream_t st) {
    return launch_f2mp_dt<STENCIL_F64>(P, src0, de, dof, k, passes, st);
}
}  // namespace sg
