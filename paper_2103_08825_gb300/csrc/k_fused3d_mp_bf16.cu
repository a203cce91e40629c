// k_fused3d_mp_bf16.cu -- instantiations of the persistent multi-pass 3D kernel for
// STENCIL_BF16 storage (own translation unit: the build compiles in parallel).
#include "k_fused3d.cuh"

namespace sg {
cudaError_t launch_f3mp_BF16(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                            cudaStream_t st) {
    return launch_f3mp_dt<STENCIL_BF16>(P, src0, de, dof, k, passes, st);
}
}  // namespace sg
