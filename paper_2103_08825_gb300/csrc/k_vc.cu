// k_vc.cu -- C ABI of the variable-coefficient sweep (kernels in k_vc.cuh):
// the pass loop over the plan's workspace, as stencil_run's.
#include <algorithm>
#include <string>

#include "k_vc.cuh"

using namespace sg;

extern "C" stencil_status_t stencil_run_vc(stencil_plan_t P, const void *coef, const void *u_in, void *u_out,
                                           int64_t T, void *stream) {
    if (!P || !coef || !u_in || !u_out || T < 0) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    if (P->dtype != STENCIL_F32 && P->dtype != STENCIL_F64 && P->dtype != STENCIL_I32) {
        set_error("variable coefficients support F32, F64 and I32 plans");
        return STENCIL_ERR_UNSUPPORTED;
    }
    const char *a = static_cast<const char *>(u_in);
    const char *b = static_cast<const char *>(u_out);
    if (a < b + P->grid_bytes && b < a + P->grid_bytes) {
        set_error("u_out must not overlap u_in");
        return STENCIL_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (T == 0) {
        cudaError_t e = cudaMemcpyAsync(u_out, u_in, P->grid_bytes, cudaMemcpyDeviceToDevice, st);
        return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    stencil_status_t s = ensure_status_word(P);
    if (s != STENCIL_OK) return s;
    // fused 2D passes of k steps (k from the plan, at most VC_KMAX), else one step per launch
    const bool fused = P->dim == 2 && P->r <= 2 && P->variant != STENCIL_VARIANT_PLAIN && !P->tuned_plain &&
                       P->n[1] + 64 < (1ll << 30) && P->n[2] + 512 < (1ll << 30);
    const int k = fused ? std::max(1, std::min(P->k > 0 ? P->k : (P->dtype == STENCIL_F64 ? 1 : 4), vc_kmax(P->r)))
                        : 1;
    const int64_t passes = (T + k - 1) / k;
    if (passes > 1) {
        s = ensure_buf(&P->ws, P->grid_bytes);
        if (s != STENCIL_OK) return s;
    }
    const void *src = u_in;
    for (int64_t p = 0; p < passes; ++p) {
        void *dst = ((passes - 1 - p) % 2 == 0) ? u_out : P->ws;
        const int kp = fused ? (int)std::min<int64_t>(k, T - p * k) : 0;
        cudaError_t e;
        switch (P->dtype) {
            case STENCIL_F32: e = launch_vc_F32(*P, kp, coef, src, dst, st); break;
            case STENCIL_F64: e = launch_vc_F64(*P, kp, coef, src, dst, st); break;
            default: e = launch_vc_I32(*P, kp, coef, src, dst, st); break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "variable-coefficient launch");
        src = dst;
    }
    return STENCIL_OK;
}
