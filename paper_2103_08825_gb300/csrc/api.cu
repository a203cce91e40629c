// api.cu -- C ABI of the stencil library: plan validation and bookkeeping,
// the pass loop of stencil_run (Section 3.3's "Main": advance k steps per
// pass until T is reached), host-buffer runs, the fusion-depth autotuner and
// status reporting.  No C++ exception crosses this boundary.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "plan.h"

namespace sg {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

size_t dtype_size(int dtype) {
    switch (dtype) {
        case STENCIL_F64: return 8;
        case STENCIL_F32: return 4;
        case STENCIL_BF16: return 2;
        case STENCIL_F16: return 2;
        case STENCIL_I32: return 4;
    }
    return 0;
}

// ------------------------------------------------------------ TMA maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool make_tmap(CUtensorMap *map, int dtype, int rank, const int64_t *dims, const uint32_t *box, const void *base) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    CUtensorMapDataType t;
    switch (dtype) {
        case STENCIL_F64: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
        case STENCIL_F32: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
        case STENCIL_BF16: t = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
        case STENCIL_F16: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
        case STENCIL_I32: t = CU_TENSOR_MAP_DATA_TYPE_INT32; break;
        default: return false;
    }
    cuuint64_t gdim[3], gstride[2];
    cuuint32_t bdim[3], estr[3] = {1, 1, 1};
    uint64_t pitch = dtype_size(dtype);
    for (int i = 0; i < rank; ++i) {
        gdim[i] = (cuuint64_t)dims[i];
        bdim[i] = box[i];
        if (i > 0) gstride[i - 1] = pitch;
        pitch *= (uint64_t)dims[i];
    }
    CUresult r = fn(map, t, (cuuint32_t)rank, const_cast<void *>(base), gdim, gstride, bdim, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------ helpers
static int npoints(int d, int r, int pattern) {
    if (pattern == STENCIL_BOX) {
        int p = 1;
        for (int a = 0; a < d; ++a) p *= 2 * r + 1;
        return p;
    }
    return 1 + 2 * d * r;
}

// Offsets in compact weight order (box lexicographic, innermost fastest;
// star [centre, axis 0: -r..-1, +1..+r, axis 1: ...]), padded to 3D.
static void compact_offsets(int d, int r, int pattern, int (*off)[3]) {
    const int np = npoints(d, r, pattern);
    for (int j = 0; j < np; ++j) off[j][0] = off[j][1] = off[j][2] = 0;
    if (pattern == STENCIL_BOX) {
        for (int j = 0; j < np; ++j) {
            int rem = j;
            for (int a = d - 1; a >= 0; --a) {
                off[j][3 - d + a] = rem % (2 * r + 1) - r;
                rem /= 2 * r + 1;
            }
        }
    } else {
        int j = 1;
        for (int a = 0; a < d; ++a)
            for (int m = -r; m <= r; ++m)
                if (m != 0) off[j++][3 - d + a] = m;
    }
}

stencil_status_t cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return STENCIL_ERR_CUDA;
}

// 32 bytes: the status word at offset 0, the per-pass kernels' job tickets at 16
stencil_status_t ensure_status_word(stencil_plan_s *P) {
    if (P->d_status) return STENCIL_OK;
    cudaError_t e = cudaMalloc(&P->d_status, 32);
    if (e != cudaSuccess) { P->d_status = nullptr; set_error("status word allocation failed"); return STENCIL_ERR_OOM; }
    e = cudaMemset(P->d_status, 0, 32);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    P->d_ctr = reinterpret_cast<char *>(P->d_status) + 16;
    return STENCIL_OK;
}

cudaError_t ensure_mp_state(const stencil_plan_s &P, int64_t tiles, cudaStream_t st) {
    if (P.d_mp && tiles <= P.mp_tiles_cap) return cudaSuccess;
    if (P.d_mp) {
        cudaFree(P.d_mp);   // synchronises the device: no launch still uses it
        P.d_mp = nullptr;
        P.mp_tiles_cap = 0;
    }
    const size_t bytes = kMpCtlBytes + sizeof(int) * (size_t)tiles;
    cudaError_t e = cudaMalloc(&P.d_mp, bytes);
    if (e != cudaSuccess) {
        P.d_mp = nullptr;
        return e;
    }
    e = cudaMemsetAsync(P.d_mp, 0, bytes, st);
    if (e != cudaSuccess) return e;
    P.mp_tiles_cap = tiles;
    return cudaSuccess;
}

stencil_status_t ensure_buf(void **buf, size_t bytes) {
    if (*buf) return STENCIL_OK;
    cudaError_t e = cudaMalloc(buf, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        *buf = nullptr;
        cudaGetLastError();
        set_error("workspace allocation of " + std::to_string(bytes) + " bytes failed");
        return STENCIL_ERR_OOM;
    }
    return STENCIL_OK;
}

static int effective_k(const stencil_plan_s *P) {
    const int km = fused_max_k(*P);
    if (km <= 0) return 1;
    int k = P->k > 0 ? P->k : std::min(km, P->dtype == STENCIL_F64 ? 1 : 4);
    return std::min(k, km);
}

static bool uses_fused(const stencil_plan_s *P) {
    return (P->variant == STENCIL_VARIANT_FUSED || P->variant == STENCIL_VARIANT_FUSED_PER_PASS) && !P->tuned_plain &&
           fused_max_k(*P) > 0;
}

// passes of exactly k steps that stencil_run gives one persistent launch
// (0: one launch per pass)
static int64_t multi_passes(const stencil_plan_s *P, int k, int64_t T) {
    if (P->variant != STENCIL_VARIANT_FUSED || !fused_multi_ok(*P, k)) return 0;
    const int64_t full = T / k;
    return full >= 2 && full <= (1 << 30) ? full : 0;
}

}  // namespace sg

using namespace sg;

extern "C" {

const char *stencil_status_string(stencil_status_t s) {
    switch (s) {
        case STENCIL_OK: return "ok";
        case STENCIL_ERR_INVALID_ARG: return "invalid argument";
        case STENCIL_ERR_UNSUPPORTED: return "unsupported";
        case STENCIL_ERR_OOM: return "out of device memory";
        case STENCIL_ERR_CUDA: return "CUDA error";
        case STENCIL_ERR_TIMEOUT: return "device-side wait timed out";
        case STENCIL_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *stencil_last_error(void) { return g_last_error.c_str(); }

stencil_status_t stencil_plan_create(stencil_plan_t *out, int32_t dim, int32_t radius, const int64_t *shape,
                                     const stencil_weights_t *weights, const stencil_boundary_t *boundary,
                                     int32_t dtype) {
    if (!out || !shape || !weights || !boundary) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    *out = nullptr;
    if (dim < 1 || dim > 3) { set_error("dim must be 1, 2 or 3"); return STENCIL_ERR_INVALID_ARG; }
    if (radius < 1 || radius > 3) { set_error("radius must be 1..3"); return STENCIL_ERR_INVALID_ARG; }
    if (weights->pattern != STENCIL_STAR && weights->pattern != STENCIL_BOX) {
        set_error("pattern must be STAR or BOX");
        return STENCIL_ERR_INVALID_ARG;
    }
    if (boundary->kind != STENCIL_DIRICHLET && boundary->kind != STENCIL_PERIODIC) {
        set_error("boundary kind must be DIRICHLET or PERIODIC");
        return STENCIL_ERR_INVALID_ARG;
    }
    if (dtype < STENCIL_F64 || dtype > STENCIL_I32) { set_error("unknown dtype"); return STENCIL_ERR_INVALID_ARG; }
    const int np = npoints(dim, radius, weights->pattern);
    if (weights->count != np || !weights->w) {
        set_error("weights.count must be " + std::to_string(np));
        return STENCIL_ERR_INVALID_ARG;
    }
    int64_t npts = 1;
    for (int a = 0; a < dim; ++a) {
        if (shape[a] < 1 || shape[a] > (int64_t(1) << 40)) { set_error("extents must be >= 1"); return STENCIL_ERR_INVALID_ARG; }
        if (npts > (int64_t(1) << 62) / shape[a]) { set_error("grid too large"); return STENCIL_ERR_INVALID_ARG; }
        npts *= shape[a];
    }
    for (int j = 0; j < np; ++j) {
        const double w = weights->w[j];
        if (!std::isfinite(w)) { set_error("weights must be finite"); return STENCIL_ERR_INVALID_ARG; }
        if (dtype == STENCIL_I32 && (w != std::floor(w) || std::fabs(w) > 9.0e15)) {
            set_error("integer mode needs integer weights");
            return STENCIL_ERR_INVALID_ARG;
        }
    }
    if (dtype == STENCIL_I32 && boundary->kind == STENCIL_DIRICHLET &&
        (boundary->value != std::floor(boundary->value) || std::fabs(boundary->value) > 9.0e15)) {
        set_error("integer mode needs an integer boundary value");
        return STENCIL_ERR_INVALID_ARG;
    }
    stencil_plan_s *P = new (std::nothrow) stencil_plan_s();
    if (!P) { set_error("host allocation failed"); return STENCIL_ERR_OOM; }
    P->dim = dim;
    P->r = radius;
    P->pattern = weights->pattern;
    P->np = np;
    P->dtype = dtype;
    P->bkind = boundary->kind;
    P->bval = boundary->kind == STENCIL_DIRICHLET ? boundary->value : 0.0;
    for (int a = 0; a < dim; ++a) P->n[3 - dim + a] = shape[a];
    P->npts = npts;
    P->grid_bytes = (size_t)npts * dtype_size(dtype);
    int off[kHostMaxPts][3];
    compact_offsets(dim, radius, weights->pattern, off);
    std::vector<int> order(np);
    for (int j = 0; j < np; ++j) { order[j] = j; P->w_compact[j] = weights->w[j]; }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        for (int c = 0; c < 3; ++c)
            if (off[a][c] != off[b][c]) return off[a][c] < off[b][c];
        return false;
    });
    for (int j = 0; j < np; ++j) {
        P->eval_to_compact[j] = order[j];
        P->w_eval[j] = weights->w[order[j]];
        for (int c = 0; c < 3; ++c) P->off_eval[j][c] = off[order[j]][c];
    }
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "no CUDA device");
    }
    // experiment overrides: STENCIL_K (fusion depth) and STENCIL_TILE (tile
    // length), applied where the kernels accept them
    if (const char *ek = getenv("STENCIL_K")) {
        const int k = atoi(ek);
        if (k >= 1 && k <= std::max(fused_max_k(*P), 1)) P->k = k;
    }
    if (const char *et = getenv("STENCIL_TILE")) {
        const int t = atoi(et);
        if (t >= 0) P->tile_rows = t;
    }
    *out = P;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_destroy(stencil_plan_t P) {
    if (!P) return STENCIL_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(P->device);
    cudaDeviceSynchronize();
    cudaFree(P->ws);
    cudaFree(P->hws[0]);
    cudaFree(P->hws[1]);
    cudaFree(P->d_status);
    cudaFree(P->adj_ws);
    cudaFree(P->vcadj_ws);
    cudaFree(P->adj_partials);
    cudaFree(P->d_mp);
    cudaFree(P->inpl_ws);
    cudaFree(P->ckpt_ws);
    for (int i = 0; i < 4; ++i) cudaFree(P->hm_buf[i]);
    if (P->hm_ready) {
        for (int i = 0; i < 2; ++i) cudaStreamDestroy(P->hm_st[i]);
        for (int i = 0; i < 7; ++i) cudaEventDestroy(P->hm_ev[i]);
    }
    cudaSetDevice(cur);
    delete P;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_set_k(stencil_plan_t P, int32_t k) {
    if (!P || k < 0) { set_error("invalid plan or k"); return STENCIL_ERR_INVALID_ARG; }
    const int km = fused_max_k(*P);
    if (k > std::max(km, 1)) {
        set_error("k=" + std::to_string(k) + " exceeds this plan's limit " + std::to_string(std::max(km, 1)));
        return STENCIL_ERR_UNSUPPORTED;
    }
    P->k = k;
    P->tuned_plain = false;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_get_k(stencil_plan_t P, int32_t *k) {
    if (!P || !k) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    if (P->variant == STENCIL_VARIANT_TESSELLATE && !P->tuned_plain) *k = P->k > 0 ? P->k : 8;   // levels per time tile
    else *k = uses_fused(P) ? effective_k(P) : 1;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_max_k(stencil_plan_t P, int32_t *kmax) {
    if (!P || !kmax) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    *kmax = std::max(fused_max_k(*P), 1);
    return STENCIL_OK;
}

stencil_status_t stencil_plan_set_variant(stencil_plan_t P, int32_t variant) {
    if (!P || (variant != STENCIL_VARIANT_FUSED && variant != STENCIL_VARIANT_PLAIN &&
               variant != STENCIL_VARIANT_FUSED_PER_PASS && variant != STENCIL_VARIANT_TESSELLATE)) {
        set_error("invalid plan or variant");
        return STENCIL_ERR_INVALID_ARG;
    }
    P->variant = variant;
    P->tuned_plain = false;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_get_variant(stencil_plan_t P, int32_t *variant) {
    if (!P || !variant) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    *variant = P->tuned_plain ? STENCIL_VARIANT_PLAIN : P->variant;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_set_tile_rows(stencil_plan_t P, int32_t rows) {
    if (!P || rows < 0) { set_error("invalid plan or tile height"); return STENCIL_ERR_INVALID_ARG; }
    P->tile_rows = rows;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_get_tile_rows(stencil_plan_t P, int32_t *rows) {
    if (!P || !rows) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    *rows = P->tile_rows;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_set_block_warps(stencil_plan_t P, int32_t warps) {
    if (!P || warps < 0 || warps > 8) { set_error("invalid plan or block size (0..8 warps)"); return STENCIL_ERR_INVALID_ARG; }
    P->block_warps = warps;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_get_block_warps(stencil_plan_t P, int32_t *warps) {
    if (!P || !warps) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    *warps = P->block_warps;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_launch_count(stencil_plan_t P, int64_t T, int64_t *launches) {
    if (!P || !launches || T < 0) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    if (T == 0) { *launches = 0; return STENCIL_OK; }
    if (P->variant == STENCIL_VARIANT_TESSELLATE && !P->tuned_plain) {
        const int h = P->k > 0 ? P->k : 8;
        *launches = 1 + (T + h - 1) / h * (P->dim + 1);   // the set-up copy, then d + 1 stages per time tile
        return STENCIL_OK;
    }
    if (!uses_fused(P)) { *launches = T; return STENCIL_OK; }
    const int k = effective_k(P);
    const int64_t mp = multi_passes(P, k, T);
    *launches = mp > 0 ? 1 + (T - mp * k > 0 ? 1 : 0) : (T + k - 1) / k;
    return STENCIL_OK;
}

stencil_status_t stencil_plan_describe(stencil_plan_t P, char *buf, int32_t len) {
    if (!P || !buf || len < 1) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    std::string s = P->variant == STENCIL_VARIANT_TESSELLATE && !P->tuned_plain
                        ? "tessellate(d+1 stages per time tile of " + std::to_string(P->k > 0 ? P->k : 8) + " levels)"
                        : uses_fused(P) ? fused_describe(*P, effective_k(P)) : std::string("plain(one step per launch)");
    strncpy(buf, s.c_str(), (size_t)len - 1);
    buf[len - 1] = 0;
    return STENCIL_OK;
}

stencil_status_t stencil_run(stencil_plan_t P, const void *u_in, void *u_out, int64_t T, void *stream) {
    if (!P || !u_in || !u_out || T < 0) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
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
    // an NVTX range around the enqueueing of the sweep (free without a tool attached)
    struct NvtxRange {
        NvtxRange() { nvtxRangePushA("stencil_run"); }
        ~NvtxRange() { nvtxRangePop(); }
    } nvtx_range;
    stencil_status_t s = ensure_status_word(P);
    if (s != STENCIL_OK) return s;
    if (P->variant == STENCIL_VARIANT_TESSELLATE && !P->tuned_plain) return tess_run(P, u_in, u_out, T, st);
    const bool fused = uses_fused(P);
    const int k = fused ? effective_k(P) : 1;
    const int64_t passes = (T + k - 1) / k;
    if (passes > 1) {
        s = ensure_buf(&P->ws, P->grid_bytes);
        if (s != STENCIL_OK) return s;
    }
    const void *src = u_in;
    int64_t p0 = 0;
    const int64_t mp = fused ? multi_passes(P, k, T) : 0;
    if (mp > 0) {
        // passes 0..mp-1 in one persistent launch; its last pass lands where
        // pass mp-1 of the loop below would
        void *de = ((passes - mp) % 2 == 0) ? u_out : P->ws;
        void *dof = de == u_out ? P->ws : u_out;
        cudaError_t e = launch_fused_multi(*P, u_in, de, dof, k, (int)mp, st);
        if (e == cudaSuccess) {
            p0 = mp;
            src = de;
        } else if (e != cudaErrorNotSupported) {
            return cuda_fail(e, "multi-pass kernel launch");
        }
    }
    for (int64_t p = p0; p < passes; ++p) {
        // the last pass lands in u_out; earlier ones alternate ws / u_out
        void *dst = ((passes - 1 - p) % 2 == 0) ? u_out : P->ws;
        const int kp = (int)std::min<int64_t>(k, T - p * k);
        cudaError_t e = fused ? launch_fused(*P, src, dst, kp, st) : launch_plain(*P, src, dst, st);
        if (e != cudaSuccess) return cuda_fail(e, fused ? "fused kernel launch" : "plain kernel launch");
        src = dst;
    }
    return STENCIL_OK;
}

stencil_status_t stencil_run_host(stencil_plan_t P, const void *h_in, void *h_out, int64_t T, void *stream) {
    if (!P || !h_in || !h_out || T < 0) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    stencil_status_t s = ensure_buf(&P->hws[0], P->grid_bytes);
    if (s == STENCIL_OK) s = ensure_buf(&P->hws[1], P->grid_bytes);
    if (s != STENCIL_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(P->hws[0], h_in, P->grid_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    s = stencil_run(P, P->hws[0], P->hws[1], T, stream);
    if (s != STENCIL_OK) return s;
    e = cudaMemcpyAsync(h_out, P->hws[1], P->grid_bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cudaStreamSynchronize");
}

stencil_status_t stencil_run_host_many(stencil_plan_t P, int64_t n, const void *const *h_in, void *const *h_out,
                                       int64_t T, void *stream) {
    if (!P || n < 0 || (n > 0 && (!h_in || !h_out)) || T < 0) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    for (int64_t i = 0; i < n; ++i)
        if (!h_in[i] || !h_out[i]) { set_error("null host buffer"); return STENCIL_ERR_INVALID_ARG; }
    if (n == 0) return STENCIL_OK;
    for (int i = 0; i < 4; ++i) {
        stencil_status_t s = ensure_buf(&P->hm_buf[i], P->grid_bytes);
        if (s != STENCIL_OK) return s;
    }
    if (!P->hm_ready) {
        for (int i = 0; i < 2; ++i)
            if (cudaStreamCreateWithFlags(&P->hm_st[i], cudaStreamNonBlocking) != cudaSuccess)
                return cuda_fail(cudaGetLastError(), "copy stream creation");
        for (int i = 0; i < 7; ++i)
            if (cudaEventCreateWithFlags(&P->hm_ev[i], cudaEventDisableTiming) != cudaSuccess)
                return cuda_fail(cudaGetLastError(), "event creation");
        P->hm_ready = true;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStream_t s_in = P->hm_st[0], s_out = P->hm_st[1];
    // events per buffer slot b: input copied (0,1), computed (2,3), output copied (4,5); 6: start
    cudaEvent_t *ev = P->hm_ev;
    cudaError_t e = cudaEventRecord(ev[6], st);   // the copies follow the caller's earlier work on `stream`
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev[6], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev[6], 0);
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    for (int64_t i = 0; i < n; ++i) {
        const int b = (int)(i & 1);
        void *din = P->hm_buf[b], *dout = P->hm_buf[2 + b];
        // input slot b is free once grid i - 2's sweep has read it
        if (i >= 2) e = cudaStreamWaitEvent(s_in, ev[2 + b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(din, h_in[i], P->grid_bytes, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(ev[b], s_in);
        // the sweep waits for its input, and for output slot b to be copied out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[b], 0);
        if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(st, ev[4 + b], 0);
        if (e != cudaSuccess) return cuda_fail(e, "pipelined host run");
        stencil_status_t s = stencil_run(P, din, dout, T, stream);
        if (s != STENCIL_OK) return s;
        e = cudaEventRecord(ev[2 + b], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev[2 + b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_out[i], dout, P->grid_bytes, cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess) e = cudaEventRecord(ev[4 + b], s_out);
        if (e != cudaSuccess) return cuda_fail(e, "pipelined host run");
    }
    // the last copies out complete before `stream` moves on; then wait
    e = cudaEventRecord(ev[6], s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[6], 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cudaStreamSynchronize");
}

// Test hook (not in the public header): sets tile `tile`'s pass counter of
// the plan's persistent multi-pass launches to a large negative value, so that
// the items of later passes that depend on it must give up their bounded
// waits -- host-side fault injection for the timeout path.  The launch's last
// worker resets every counter to zero as usual.  The counters must exist (a
// persistent launch has run) and no launch of the plan may be in flight.
stencil_status_t stencil_plan_test_poison_counter(stencil_plan_t P, int64_t tile) {
    if (!P || tile < 0) return STENCIL_ERR_INVALID_ARG;
    if (!P->d_mp || tile >= P->mp_tiles_cap) return STENCIL_ERR_INVALID_ARG;
    const int v = -(1 << 30);
    int *done = reinterpret_cast<int *>(static_cast<char *>(P->d_mp) + kMpCtlBytes);
    if (cudaMemcpy(done + tile, &v, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return STENCIL_ERR_CUDA;
    return STENCIL_OK;
}

stencil_status_t stencil_get_device_status(stencil_plan_t P) {
    if (!P) { set_error("null plan"); return STENCIL_ERR_INVALID_ARG; }
    if (!P->d_status) return STENCIL_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    int h = 0;
    e = cudaMemcpy(&h, P->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (h != 0) {
        cudaMemset(P->d_status, 0, sizeof(int));
        set_error("a device-side bounded wait gave up");
        return (stencil_status_t)h;
    }
    return STENCIL_OK;
}

}  // extern "C"
