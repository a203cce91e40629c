// k_plain_i32.cu -- the one-step sweep kernels for I32 storage.
#include "k_plain.cuh"

namespace sg {
cudaError_t launch_plain_I32(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    return plain_dispatch_d<STENCIL_I32>(P, src, dst, st);
}
}  // namespace sg
