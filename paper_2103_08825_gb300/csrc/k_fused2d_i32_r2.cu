// k_fused2d_i32_r2.cu -- instantiations of the 2D fused kernel for
// STENCIL_I32 storage, radius 2 (own translation unit: the build compiles in parallel).
#include "k_fused2d.cuh"

namespace sg {
template cudaError_t launch_f2_range<STENCIL_I32, 2, 1, 16>(const stencil_plan_s &, const void *, void *, int,
                                                             cudaStream_t);
}  // namespace sg
