// k_fused2d_mp_i32_r1hi.cu -- instantiations of the persistent multi-pass 2D
// kernel for STENCIL_I32 storage, radius 1, fusion depths 9..16 (own translation unit: the build
// compiles in parallel).
#include "k_fused2d.cuh"

namespace sg {
template cudaError_t launch_f2mp_range<STENCIL_I32, 1, 9, 16>(const stencil_plan_s &, const void *, void *,
                                                               void *, int, int, cudaStream_t);
}  // namespace sg
