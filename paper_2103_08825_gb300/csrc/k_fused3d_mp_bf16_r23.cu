// k_fused3d_mp_bf16_r23.cu -- the persistent multi-pass 3D kernel for
// STENCIL_BF16 storage, radii 2 and 3 (own translation unit: the build compiles
// in parallel).
#include "k_fused3d.cuh"

namespace sg {
template cudaError_t launch_f3mp_r<STENCIL_BF16, 2>(const stencil_plan_s &, const void *, void *, void *, int, int,
                                                    cudaStream_t);
template cudaError_t launch_f3mp_r<STENCIL_BF16, 3>(const stencil_plan_s &, const void *, void *, void *, int, int,
                                                    cudaStream_t);
}  // namespace sg
