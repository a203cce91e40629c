// k_inplace2d_i32.cu -- the in-place 2D sweep for STENCIL_I32 storage.
#include "k_inplace2d.cuh"

namespace sg {
cudaError_t launch_inpl_I32(const stencil_plan_s &P, int k, void *u, const void *ri, void *ro, const InplGeo &t,
                           cudaStream_t st) {
    return launch_inpl_dt<STENCIL_I32>(P, k, u, ri, ro, t, st);
}
cudaError_t launch_inpl_init_I32(const void *u, void *ring, const InplGeo &t, int sm_count, cudaStream_t st) {
    return launch_inpl_init_dt<STENCIL_I32>(u, ring, t, sm_count, st);
}
}  // namespace sg
