// k_plain_f64.cu -- the one-step sweep kernels for F64 storage.
#include "k_plain.cuh"

namespace sg {
cudaError_t launch_plain_F64(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    return plain_dispatch_d<STENCIL_F64>(P, src, dst, st);
}
}  // namespace sg
