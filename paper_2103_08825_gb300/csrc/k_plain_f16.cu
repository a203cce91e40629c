// k_plain_f16.cu -- the one-step sweep kernels for F16 storage.
#include "k_plain.cuh"

namespace sg {
cudaError_t launch_plain_F16(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    return plain_dispatch_d<STENCIL_F16>(P, src, dst, st);
}
}  // namespace sg
