// k_inplace2d.cu -- C ABI of the in-place 2D sweep (kernels in
// k_inplace2d.cuh): ring set-up, the pass loop, and the workspace query.
#include <algorithm>
#include <string>

#include "k_inplace2d.cuh"

namespace sg {

static int inpl_k(const stencil_plan_s &P) {
    const int k = P.k > 0 ? P.k : (P.dtype == STENCIL_F64 ? 1 : 4);
    return std::max(1, std::min(k, inpl_kmax(P.r)));
}

static size_t inpl_bytes(const stencil_plan_s &P, const InplGeo &t) {
    return 2 * (size_t)t.bands * t.chunks * t.ring * dtype_size(P.dtype);
}

static cudaError_t inpl_launch(const stencil_plan_s &P, int k, void *u, const void *ri, void *ro, const InplGeo &t,
                               cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F32: return launch_inpl_F32(P, k, u, ri, ro, t, st);
        case STENCIL_F64: return launch_inpl_F64(P, k, u, ri, ro, t, st);
        case STENCIL_BF16: return launch_inpl_BF16(P, k, u, ri, ro, t, st);
        case STENCIL_F16: return launch_inpl_F16(P, k, u, ri, ro, t, st);
        case STENCIL_I32: return launch_inpl_I32(P, k, u, ri, ro, t, st);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t inpl_init(const stencil_plan_s &P, const void *u, void *ring, const InplGeo &t, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F32: return launch_inpl_init_F32(u, ring, t, P.sm_count, st);
        case STENCIL_F64: return launch_inpl_init_F64(u, ring, t, P.sm_count, st);
        case STENCIL_BF16: return launch_inpl_init_BF16(u, ring, t, P.sm_count, st);
        case STENCIL_F16: return launch_inpl_init_F16(u, ring, t, P.sm_count, st);
        case STENCIL_I32: return launch_inpl_init_I32(u, ring, t, P.sm_count, st);
    }
    return cudaErrorInvalidValue;
}

static stencil_status_t inpl_check(const stencil_plan_s *P) {
    if (P->dim != 2) {
        set_error("the in-place sweep supports 2D plans");
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (P->n[1] + 64 >= (1ll << 30) || P->n[2] + 512 >= (1ll << 30)) {
        set_error("the in-place sweep keeps 32-bit indices: extents below 2^30");
        return STENCIL_ERR_UNSUPPORTED;
    }
    return STENCIL_OK;
}

}  // namespace sg

using namespace sg;

extern "C" stencil_status_t stencil_inplace_workspace_bytes(stencil_plan_t P, int64_t *bytes) {
    if (!P || !bytes) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    stencil_status_t s = inpl_check(P);
    if (s != STENCIL_OK) return s;
    *bytes = (int64_t)inpl_bytes(*P, inpl_geo(*P, inpl_k(*P)));
    return STENCIL_OK;
}

extern "C" stencil_status_t stencil_run_inplace(stencil_plan_t P, void *u, int64_t T, void *stream) {
    if (!P || !u || T < 0) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    stencil_status_t s = inpl_check(P);
    if (s != STENCIL_OK) return s;
    if (T == 0) return STENCIL_OK;
    s = ensure_status_word(P);
    if (s != STENCIL_OK) return s;
    const int k = inpl_k(*P);
    const InplGeo t = inpl_geo(*P, k);
    const size_t need = inpl_bytes(*P, t);
    if (P->inpl_ws_bytes < need) {
        cudaFree(P->inpl_ws);   // synchronises the device: no launch still uses it
        P->inpl_ws = nullptr;
        P->inpl_ws_bytes = 0;
        if (cudaMalloc(&P->inpl_ws, need) != cudaSuccess) {
            cudaGetLastError();
            set_error("in-place ring allocation of " + std::to_string(need) + " bytes failed");
            return STENCIL_ERR_OOM;
        }
        P->inpl_ws_bytes = need;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ring[2] = {static_cast<char *>(P->inpl_ws), static_cast<char *>(P->inpl_ws) + need / 2};
    cudaError_t e = inpl_init(*P, u, ring[0], t, st);
    if (e != cudaSuccess) return cuda_fail(e, "in-place ring set-up");
    const int64_t passes = (T + k - 1) / k;
    for (int64_t p = 0; p < passes; ++p) {
        const int kp = (int)std::min<int64_t>(k, T - p * k);
        e = inpl_launch(*P, kp, u, ring[p & 1], ring[(p + 1) & 1], t, st);
        if (e != cudaSuccess) return cuda_fail(e, "in-place pass launch");
    }
    return STENCIL_OK;
}
