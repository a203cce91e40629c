// k_plain_bf16.cu -- the one-step sweep kernels for BF16 storage.
#include "k_plain.cuh"

namespace sg {
cudaError_t launch_plain_BF16(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    return plain_dispatch_d<STENCIL_BF16>(P, src, dst, st);
}
}  // namespace sg
