// k_fused3d_f16.cu -- instantiations of the 3D fused kernel for STENCIL_F16
// storage (one translation unit per dtype keeps the build parallel).
#include "k_fused3d.cuh"

namespace sg {
cudaError_t launch_f3_F16(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f3_dt<STENCIL_F16>(P, src, dst, k, st);
}
}  // namespace sg
