// k_plain.cu -- dispatch of the one-step sweep to the translation unit of the
// plan's storage type (k_plain_<dtype>.cu; kernels in k_plain.cuh).
#include "k_plain.cuh"

namespace sg {

cudaError_t launch_plain(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F64: return launch_plain_F64(P, src, dst, st);
        case STENCIL_F32: return launch_plain_F32(P, src, dst, st);
        case STENCIL_BF16: return launch_plain_BF16(P, src, dst, st);
        case STENCIL_F16: return launch_plain_F16(P, src, dst, st);
        case STENCIL_I32: return launch_plain_I32(P, src, dst, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sg
