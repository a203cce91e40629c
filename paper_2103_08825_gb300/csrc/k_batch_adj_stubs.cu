// k_batch_adj_stubs.cu -- entry points whose kernels are not built yet.
#include "plan.h"

using namespace sg;

extern "C" {

stencil_status_t stencil_batch_create(stencil_batch_t *out, int32_t, int32_t, int32_t, const int64_t *,
                                      const stencil_weights_t *, const int64_t *, const stencil_boundary_t *, int32_t) {
    if (out) *out = nullptr;
    set_error("batched runs are not available in this build");
    return STENCIL_ERR_UNSUPPORTED;
}
stencil_status_t stencil_batch_destroy(stencil_batch_t) { return STENCIL_OK; }
stencil_status_t stencil_batch_run(stencil_batch_t, const void *const *, void *const *, void *) {
    set_error("batched runs are not available in this build");
    return STENCIL_ERR_UNSUPPORTED;
}
stencil_status_t stencil_batch_get_device_status(stencil_batch_t) { return STENCIL_ERR_UNSUPPORTED; }
stencil_status_t stencil_batch_launch_count(stencil_batch_t, int64_t *) { return STENCIL_ERR_UNSUPPORTED; }

stencil_status_t stencil_adjoint_run(stencil_plan_t, const void *, const void *, int64_t, int32_t, void *, double *,
                                     void *) {
    set_error("the adjoint is not available in this build");
    return STENCIL_ERR_UNSUPPORTED;
}

}  // extern "C"
