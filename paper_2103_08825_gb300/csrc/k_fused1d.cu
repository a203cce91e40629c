// k_fused1d.cu -- dispatch of the 1D fused sweep (kernels in k_fused1d.cuh,
// instantiated per storage type in k_fused1d_<dtype>.cu).
#include "k_fused1d.cuh"

namespace sg {

// The persistent form wraps a periodic halo at most once (n >= 2 chunks) and
// keeps element indices in 32 bits.
bool fused1d_multi_ok(const stencil_plan_s &P, int k) {
    if (P.dim != 1 || k < 1 || k > fused1d_max_k(P)) return false;
    const int64_t cw = 32 * (P.dtype == STENCIL_F64 ? 2 : 4);
    if (P.n[2] + 4 * cw >= (1ll << 30)) return false;
    if (P.bkind == STENCIL_PERIODIC && P.n[2] < 2 * cw) return false;
    return true;
}

cudaError_t launch_fused1d_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                                 int passes, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F64: return launch_f1mp_F64(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_F32: return launch_f1mp_F32(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_BF16: return launch_f1mp_BF16(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_F16: return launch_f1mp_F16(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_I32: return launch_f1mp_I32(P, src0, dst_even, dst_odd, k, passes, st);
    }
    return cudaErrorInvalidValue;
}

int fused1d_max_k(const stencil_plan_s &P) {
    if (P.dim != 1 || P.r > 3) return 0;
    return (P.dtype == STENCIL_BF16 || P.dtype == STENCIL_F16) ? 8 : F1_KMAX;
}

cudaError_t launch_fused1d(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F64: return launch_f1_F64(P, src, dst, k, st);
        case STENCIL_F32: return launch_f1_F32(P, src, dst, k, st);
        case STENCIL_BF16: return launch_f1_BF16(P, src, dst, k, st);
        case STENCIL_F16: return launch_f1_F16(P, src, dst, k, st);
        case STENCIL_I32: return launch_f1_I32(P, src, dst, k, st);
    }
    return cudaErrorInvalidValue;
}

std::string fused1d_describe(const stencil_plan_s &P, int k) {
    return "fused1d(warp-streamed vector sets, k=" + std::to_string(k) + ")";
}

}  // namespace sg
