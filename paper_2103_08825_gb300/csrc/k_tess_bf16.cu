// k_tess_bf16.cu -- the tessellate-tiling kernels for STENCIL_BF16 storage.
#include "k_tess.cuh"

namespace sg {
cudaError_t launch_tess_BF16(const stencil_plan_s &P, const TessGeo &geo, void *b0, void *b1, int t0, int hlev,
                           cudaStream_t st) {
    return launch_tess_dt<STENCIL_BF16>(P, geo, b0, b1, t0, hlev, st);
}
}  // namespace sg
