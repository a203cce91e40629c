// k_fused3d_mp_bf16.cu -- the persistent multi-pass 3D kernel for STENCIL_BF16
// storage, radius 1, and its dispatcher (radii 2 and 3: k_fused3d_mp_bf16_r23.cu).
#include "k_fused3d.cuh"

namespace sg {
extern template cudaError_t launch_f3mp_r<STENCIL_BF16, 2>(const stencil_plan_s &, const void *, void *, void *, int,
                                                           int, cudaStream_t);
extern template cudaError_t launch_f3mp_r<STENCIL_BF16, 3>(const stencil_plan_s &, const void *, void *, void *, int,
                                                           int, cudaStream_t);
cudaError_t launch_f3mp_BF16(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                            cudaStream_t st) {
    return launch_f3mp_dt<STENCIL_BF16>(P, src0, de, dof, k, passes, st);
}
}  // namespace sg
