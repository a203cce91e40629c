// k_fused2d_f64.cu -- the 2D fused kernel for STENCIL_F64 storage: radius 1
// at fusion depths 1..8, and the dispatcher.  Radii 2 and 3 are instantiated
// in k_fused2d_f64_r2.cu and _r3.cu (one translation unit each keeps the build
// parallel); depths above 8 exist only as the persistent kernel.
#include "k_fused2d.cuh"

namespace sg {
extern template cudaError_t launch_f2_range<STENCIL_F64, 2, 1, 16>(const stencil_plan_s &, const void *, void *,
                                                                    int, cudaStream_t);
extern template cudaError_t launch_f2_range<STENCIL_F64, 3, 1, 16>(const stencil_plan_s &, const void *, void *,
                                                                    int, cudaStream_t);
cudaError_t launch_f2_F64(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f2_dt<STENCIL_F64>(P, src, dst, k, st);
}
int f2_kmax_F64(int r) { return f2_kmax<STENCIL_F64>(r); }
// output columns of a band: the 32 V-wide window less an aligned halo each side
int f2_bw_F64(int r, int k) {
    const int v = Traits<STENCIL_F64>::V, w = 32 * v;
    const int al = align_elems<STENCIL_F64>() > v ? align_elems<STENCIL_F64>() : v;
    return w - 2 * ((r * k + al - 1) / al * al);
}
}  // namespace sg
