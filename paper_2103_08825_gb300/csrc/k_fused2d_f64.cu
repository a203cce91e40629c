// k_fused2d_f64.cu -- instantiations of the 2D fused kernel for STENCIL_F64
// storage, radius 1, and the dispatcher (radius 2 is instantiated in
// k_fused2d_f64_r2.cu: one translation unit each keeps the build parallel).
#include "k_fused2d.cuh"

namespace sg {
extern template cudaError_t launch_f2_r<STENCIL_F64, 2>(const stencil_plan_s &, const void *, void *, int,
                                                          cudaStream_t);
cudaError_t launch_f2_F64(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f2_dt<STENCIL_F64>(P, src, dst, k, st);
}
int f2_kmax_F64(int r) { return f2_kmax<STENCIL_F64>(r); }
int f2_bw_F64(int r, int k) {
    switch (k) {
        case 1: return r == 1 ? F2Geo<STENCIL_F64, 1, 1>::BW : F2Geo<STENCIL_F64, 2, 1>::BW;
        case 2: return r == 1 ? F2Geo<STENCIL_F64, 1, 2>::BW : F2Geo<STENCIL_F64, 2, 2>::BW;
        default: {
            int v = Traits<STENCIL_F64>::V, w = 32 * v, al = align_elems<STENCIL_F64>() > v ? align_elems<STENCIL_F64>() : v;
            int h = (r * k + al - 1) / al * al;
            return w - 2 * h;
        }
    }
}
}  // namespace sg
