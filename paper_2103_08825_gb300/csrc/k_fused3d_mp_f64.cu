// k_fused3d_mp_f64.cu -- instantiations of the persistent multi-pass 3D kernel for
// STENCIL_F64 storage (own translation unit: the build compiles in parallel).
#include "k_fused3d.cuh"

namespace sg {
cudaError_t launch_f3mp_F64(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                            cudaStream_t st) {
    return launch_f3mp_dt<STENCIL_F64>(P, src0, de, dof, k, passes, st);
}
}  // namespace sg
