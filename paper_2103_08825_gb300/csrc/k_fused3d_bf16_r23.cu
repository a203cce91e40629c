// k_fused3d_bf16_r23.cu -- the 3D fused kernel for STENCIL_BF16 storage, radii 2
// and 3 (own translation unit: the build compiles in parallel).
#include "k_fused3d.cuh"

namespace sg {
template cudaError_t launch_f3_r<STENCIL_BF16, 2>(const stencil_plan_s &, const void *, void *, int, cudaStream_t);
template cudaError_t launch_f3_r<STENCIL_BF16, 3>(const stencil_plan_s &, const void *, void *, int, cudaStream_t);
}  // namespace sg
