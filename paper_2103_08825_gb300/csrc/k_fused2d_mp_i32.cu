// k_fused2d_mp_i32.cu -- the persistent multi-pass 2D kernel for STENCIL_I32
// storage: radius 1 at fusion depths 1..8, and its dispatcher (depths 9..16
// and radii 2, 3: k_fused2d_mp_i32_r1hi.cu, _r2.cu, _r3.cu).
#include "k_fused2d.cuh"

namespace sg {
extern template cudaError_t launch_f2mp_range<STENCIL_I32, 1, 9, 16>(const stencil_plan_s &, const void *, void *,
                                                                      void *, int, int, cudaStream_t);
extern template cudaError_t launch_f2mp_range<STENCIL_I32, 2, 1, 16>(const stencil_plan_s &, const void *, void *,
                                                                      void *, int, int, cudaStream_t);
extern template cudaError_t launch_f2mp_range<STENCIL_I32, 3, 1, 16>(const stencil_plan_s &, const void *, void *,
                                                                      void *, int, int, cudaStream_t);
cudaError_t launch_f2mp_I32(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                            cudaStream_t st) {
    return launch_f2mp_dt<STENCIL_I32>(P, src0, de, dof, k, passes, st);
}
}  // namespace sg
