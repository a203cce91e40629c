// k_inplace2d_f64.cu -- the in-place 2D sweep for STENCIL_F64 storage.
#include "k_inplace2d.cuh"

namespace sg {
cudaError_t launch_inpl_F64(const stencil_plan_s &P, int k, void *u, const void *ri, void *ro, const InplGeo &t,
                           cudaStream_t st) {
    return launch_inpl_dt<STENCIL_F64>(P, k, u, ri, ro, t, st);
}
cudaError_t launch_inpl_init_F64(const void *u, void *ring, const InplGeo &t, int sm_count, cudaStream_t st) {
    return launch_inpl_init_dt<STENCIL_F64>(u, ring, t, sm_count, st);
}
}  // namespace sg
