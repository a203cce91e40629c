// k_fused2d_bf16.cu -- instantiations of the 2D fused kernel for STENCIL_BF16
// storage, radius 1, and the dispatcher (radius 2 is instantiated in
// k_fused2d_bf16_r2.cu: one translation unit each keeps the build parallel).
#include "k_fused2d.cuh"

namespace sg {
extern template cudaError_t launch_f2_r<STENCIL_BF16, 2>(const stencil_plan_s &, const void *, void *, int,
                                                          cudaStream_t);
cudaError_t launch_f2_BF16(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f2_dt<STENCIL_BF16>(P, src, dst, k, st);
}
int f2_kmax_BF16(int r) { return f2_kmax<STENCIL_BF16>(r); }
int f2_bw_BF16(int r, int k) {
    switch (k) {
        case 1: return r == 1 ? F2Geo<STENCIL_BF16, 1, 1>::BW : F2Geo<STENCIL_BF16, 2, 1>::BW;
        case 2: return r == 1 ? F2Geo<STENCIL_BF16, 1, 2>::BW : F2Geo<STENCIL_BF16, 2, 2>::BW;
        default: {
            int v = Traits<STENCIL_BF16>::V, w = 32 * v, al = align_elems<STENCIL_BF16>() > v ? align_elems<STENCIL_BF16>() : v;
            int h = (r * k + al - 1) / al * al;
            return w - 2 * h;
        }
    }
}
}  // namespace sg
