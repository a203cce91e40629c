// tune.cu -- the autotuner of the fused sweep: fusion depth k (the paper's
// unrolling factor, Section 3.3, chosen here by measurement instead of by the
// register count of Section 3.3's last paragraph), launch form, tile length
// and block size, with a persistent cache of the choices.
//
// Search: stencil_run is timed with CUDA events on plan-owned buffers for
// the one-step kernel and for every supported k with one launch per pass and
// with the persistent multi-pass launch at a few tile lengths; the fastest
// then gets a second stage over the 2D kernels' block sizes (2, 4, 8 warps).
//
// Cache: one line per tuned configuration in a text file -- the path in
// STENCIL_TUNE_CACHE, else $HOME/.cache/stencil_gb300/tune.txt; the value
// "off" disables it.  The key names the device (name, SM count), the library
// build, the dimension, radius, pattern, storage type, boundary kind, the
// extents rounded up to a multiple of 64 and T.  A later stencil_plan_tune of
// a matching plan applies the stored choice without timing anything.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <sys/stat.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

namespace sg {

namespace {

std::mutex g_cache_mu;

std::string cache_path() {
    const char *p = getenv("STENCIL_TUNE_CACHE");
    if (p && *p) return std::string(p) == "off" ? std::string() : std::string(p);
    const char *home = getenv("HOME");
    if (!home || !*home) return std::string();
    return std::string(home) + "/.cache/stencil_gb300/tune.txt";
}

int64_t bucket(int64_t n) { return n <= 64 ? n : (n + 63) / 64 * 64; }

std::string cache_key(const stencil_plan_s &P, int64_t T) {
    cudaDeviceProp prop;
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&prop, P.device) == cudaSuccess) dev = prop.name;
    for (char &c : dev)
        if (c == ' ' || c == '\t') c = '_';
    std::string build = std::string(__DATE__ "_" __TIME__);
    for (char &c : build)
        if (c == ' ' || c == ':') c = '_';
    char buf[512];
    snprintf(buf, sizeof(buf), "%s/sm%d/%s/d%d/r%d/p%d/t%d/b%d/%lldx%lldx%lld/T%lld", dev.c_str(), P.sm_count,
             build.c_str(), P.dim, P.r, P.pattern, P.dtype, P.bkind, (long long)bucket(P.n[0]),
             (long long)bucket(P.n[1]), (long long)bucket(P.n[2]), (long long)T);
    return buf;
}

struct Choice {
    int k, variant, rows, warps, plain;
    double ms;
};

bool cache_lookup(const std::string &key, Choice &c) {
    const std::string path = cache_path();
    if (path.empty()) return false;
    std::lock_guard<std::mutex> lock(g_cache_mu);
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[600];
        Choice t;
        if (sscanf(line, "%599s %d %d %d %d %d %lf", k, &t.k, &t.variant, &t.rows, &t.warps, &t.plain, &t.ms) == 7 &&
            key == k) {
            c = t;   // the last matching line wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const std::string &key, const Choice &c) {
    const std::string path = cache_path();
    if (path.empty()) return;
    std::lock_guard<std::mutex> lock(g_cache_mu);
    // create the directory chain of the default location (a path given in
    // STENCIL_TUNE_CACHE must name an existing directory)
    if (!getenv("STENCIL_TUNE_CACHE")) {
        const size_t slash = path.rfind('/');
        for (size_t i = 1; slash != std::string::npos && i <= slash; ++i)
            if (i == slash || path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
    }
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %.6f\n", key.c_str(), c.k, c.variant, c.rows, c.warps, c.plain, c.ms);
    fclose(f);
}

void apply(stencil_plan_s *P, const Choice &c) {
    P->k = c.k;
    P->variant = c.variant;
    P->tile_rows = c.rows;
    P->block_warps = c.warps;
    P->tuned_plain = c.plain != 0;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" stencil_status_t stencil_plan_tune(stencil_plan_t P, int64_t T, void *stream, int32_t *best_k,
                                              double *best_ms) {
    if (!P || T < 1) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    const int km = fused_max_k(*P);
    if (km <= 0 || P->variant == STENCIL_VARIANT_PLAIN) {
        if (best_k) *best_k = 1;
        if (best_ms) *best_ms = -1.0;
        return STENCIL_OK;
    }
    const std::string key = cache_key(*P, T);
    Choice c;
    if (cache_lookup(key, c) && c.k >= 1 && c.k <= km) {
        apply(P, c);
        if (best_k) *best_k = c.plain ? 0 : c.k;
        if (best_ms) *best_ms = c.ms;
        return STENCIL_OK;
    }
    stencil_status_t s = ensure_buf(&P->hws[0], P->grid_bytes);
    if (s == STENCIL_OK) s = ensure_buf(&P->hws[1], P->grid_bytes);
    if (s != STENCIL_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(P->hws[0], 0, P->grid_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Choice saved{P->k, P->variant, P->tile_rows, P->block_warps, P->tuned_plain ? 1 : 0, 0.0};
    Choice best = saved;
    best.ms = 1e30;
    // best of three timed runs after one warm-up; false on an error (s set)
    auto time_it = [&](const Choice &cand, double &ms_out) -> bool {
        apply(P, cand);
        s = stencil_run(P, P->hws[0], P->hws[1], T, stream);
        if (s != STENCIL_OK) return false;
        float bms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            s = stencil_run(P, P->hws[0], P->hws[1], T, stream);
            cudaEventRecord(e1, st);
            if (s != STENCIL_OK) return false;
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { s = cuda_fail(e, "tuning run"); return false; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            bms = std::min(bms, ms);
        }
        ms_out = bms;
        return true;
    };
    // tile lengths: the default and a few fixed lengths below the extent
    std::vector<int> rows_c = {0};
    if (P->dim == 2)
        for (int r : {32, 48, 64, 96, 128, 192})
            if (r < P->n[1]) rows_c.push_back(r);
    if (P->dim == 3)
        for (int r : {16, 32, 48, 64, 96, 128, 192})
            if (r < P->n[0]) rows_c.push_back(r);
    if (P->dim == 1)
        for (int r : {2, 4, 8, 16, 32})
            if (r * 128 < P->n[2]) rows_c.push_back(r);
    // stage 1: k = 0 is the one-step kernel; then every fused depth, one
    // launch per pass (default tiles) and, where the grid allows it, the
    // persistent launch at each tile length
    for (int k = 0; k <= km && s == STENCIL_OK; ++k) {
        std::vector<Choice> cands;
        if (k == 0) {
            cands.push_back({1, saved.variant, saved.rows, saved.warps, 1, 0.0});
        } else {
            cands.push_back({k, STENCIL_VARIANT_FUSED_PER_PASS, 0, 0, 0, 0.0});
            if (fused_multi_ok(*P, k))
                for (int r : rows_c) cands.push_back({k, STENCIL_VARIANT_FUSED, r, 0, 0, 0.0});
        }
        for (const Choice &cand : cands) {
            double ms = 0.0;
            if (!time_it(cand, ms)) break;
            if (ms < best.ms) {
                best = cand;
                best.ms = ms;
            }
        }
    }
    // stage 2: block size of the 2D fused kernels around the best choice
    if (s == STENCIL_OK && P->dim == 2 && !best.plain) {
        const Choice base = best;
        for (int w : {2, 8}) {
            Choice cand = base;
            cand.warps = w;
            double ms = 0.0;
            if (!time_it(cand, ms)) break;
            if (ms < best.ms) {
                best = cand;
                best.ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != STENCIL_OK) {
        apply(P, saved);
        return s;
    }
    if (best.plain) {   // keep the caller's launch settings for the fused kernels
        best.variant = saved.variant;
        best.rows = saved.rows;
        best.warps = saved.warps;
    }
    apply(P, best);
    cache_store(key, best);
    if (best_k) *best_k = best.plain ? 0 : best.k;
    if (best_ms) *best_ms = best.ms;
    return STENCIL_OK;
}
