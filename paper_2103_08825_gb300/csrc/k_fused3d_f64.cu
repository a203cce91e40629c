// k_fused3d_f64.cu -- the 3D fused kernel for STENCIL_F64 storage, radius 1,
// and its dispatcher (radii 2 and 3: k_fused3d_f64_r23.cu; one translation
// unit each keeps the build parallel).
#include "k_fused3d.cuh"

namespace sg {
extern template cudaError_t launch_f3_r<STENCIL_F64, 2>(const stencil_plan_s &, const void *, void *, int,
                                                         cudaStream_t);
extern template cudaError_t launch_f3_r<STENCIL_F64, 3>(const stencil_plan_s &, const void *, void *, int,
                                                         cudaStream_t);
cudaError_t launch_f3_F64(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f3_dt<STENCIL_F64>(P, src, dst, k, st);
}
}  // namespace sg
