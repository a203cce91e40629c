// k_fused2d_mp_f32_r3.cu -- instantiations of the persistent multi-pass 2D
// kernel for STENCIL_F32 storage, radius 3 (own translation unit: the build
// compiles in parallel).
#include "k_fused2d.cuh"

namespace sg {
template cudaError_t launch_f2mp_range<STENCIL_F32, 3, 1, 16>(const stencil_plan_s &, const void *, void *,
                                                               void *, int, int, cudaStream_t);
}  // namespace sg
