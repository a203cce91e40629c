// k_adj_stub.cu -- the adjoint entry point, not built yet.
#include "plan.h"

using namespace sg;

extern "C" {

stencil_status_t stencil_adjoint_run(stencil_plan_t, const void *, const void *, int64_t, int32_t, void *, double *,
                                     void *) {
    set_error("the adjoint is not available in this build");
    return STENCIL_ERR_UNSUPPORTED;
}

}  // extern "C"
