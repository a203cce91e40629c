// k_stubs.cu -- dimensions without a fused kernel yet: max_k = 0 makes
// stencil_run use the plain one-step kernel for them (1D).
#include <string>

#include "plan.h"

namespace sg {

int fused1d_max_k(const stencil_plan_s &) { return 0; }
cudaError_t launch_fused1d(const stencil_plan_s &, const void *, void *, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
std::string fused1d_describe(const stencil_plan_s &, int) { return "none"; }



}  // namespace sg
