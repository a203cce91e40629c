// k_tess.cu -- the tessellate-tiling sweep (kernels in k_tess.cuh): geometry,
// the time-tile / stage loop, and a host-only query of the per-point level
// counts of every stage (the state sequences of the paper's Fig. 6).
#include <algorithm>
#include <string>
#include <vector>

#include "k_tess.cuh"

namespace sg {

// default segment length by dimension (at least 2 h r)
// default segment length: 2048, 64, 16 points in 1D, 2D, 3D -- the 3D tile's
// two level buffers then fit in shared memory (16^3 points)
static int tess_default_b(int d) { return d == 1 ? 2048 : d == 2 ? 64 : 16; }

// Axes for extents n (outermost first, d of them), tile length b, h levels,
// radius r; false if some segment is shorter than 2 h r.
static bool tess_geo(int d, const int64_t *n, int b, int h, int r, bool periodic, TessGeo &g) {
    g.d = d;
    g.h = h;
    g.r = r;
    for (int a = 0; a < 3; ++a) g.ax[a] = TessAxis{1, 1, 1, 0};
    for (int a = 0; a < d; ++a) {
        TessAxis &x = g.ax[3 - d + a];
        x.n = (int)n[a];
        x.b = std::max(1, std::min(b, x.n));
        x.m = x.n < 2 * x.b ? 1 : x.n / x.b;
        x.periodic = periodic ? 1 : 0;
        const int wmin = x.m == 1 ? x.n : x.b;
        if (wmin < 2 * h * r) return false;
    }
    return true;
}

static cudaError_t tess_launch(const stencil_plan_s &P, const TessGeo &g, void *b0, void *b1, int t0, int hl,
                               cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F32: return launch_tess_F32(P, g, b0, b1, t0, hl, st);
        case STENCIL_F64: return launch_tess_F64(P, g, b0, b1, t0, hl, st);
        case STENCIL_BF16: return launch_tess_BF16(P, g, b0, b1, t0, hl, st);
        case STENCIL_F16: return launch_tess_F16(P, g, b0, b1, t0, hl, st);
        case STENCIL_I32: return launch_tess_I32(P, g, b0, b1, t0, hl, st);
    }
    return cudaErrorInvalidValue;
}

// T steps by tessellation: time tiles of h = the plan's k levels (default 8),
// segments of the plan's tile length (default by dimension, at least 2 h r);
// the levels alternate between u_out and the plan's workspace grid so that
// level T lands in u_out.
stencil_status_t tess_run(stencil_plan_s *P, const void *u_in, void *u_out, int64_t T, cudaStream_t st) {
    const int h = P->k > 0 ? P->k : 8;
    const int b = std::max(P->tile_rows > 0 ? P->tile_rows : tess_default_b(P->dim), 2 * h * P->r);
    TessGeo g;
    if (P->n[0] >= (1ll << 30) || P->n[1] >= (1ll << 30) || P->n[2] >= (1ll << 30) ||
        !tess_geo(P->dim, P->n + (3 - P->dim), b, h, P->r, P->bkind == STENCIL_PERIODIC, g)) {
        set_error("tessellation needs every extent >= 2 h r (h = the plan's k)");
        return STENCIL_ERR_UNSUPPORTED;
    }
    // a tile (segments shorter than 2b, or the whole axis) indexes its points in 32 bits
    int64_t tile_pts = 1;
    for (int a = 0; a < 3; ++a) tile_pts *= std::min<int64_t>(g.ax[a].n, 2 * (int64_t)g.ax[a].b);
    if (tile_pts >= (1ll << 31)) {
        set_error("tessellation tile too large (tile extent^d must stay below 2^31 points)");
        return STENCIL_ERR_UNSUPPORTED;
    }
    stencil_status_t s = ensure_buf(&P->ws, P->grid_bytes);
    if (s != STENCIL_OK) return s;
    void *buf[2];
    buf[T & 1] = u_out;
    buf[(T + 1) & 1] = P->ws;
    cudaError_t e = cudaMemcpyAsync(buf[0], u_in, P->grid_bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "tessellation set-up copy");
    for (int64_t t0 = 0; t0 < T; t0 += h) {
        const int hl = (int)std::min<int64_t>(h, T - t0);
        for (int stage = 0; stage <= P->dim; ++stage) {
            tess_stage(g, stage);
            e = tess_launch(*P, g, buf[0], buf[1], (int)(t0 & 1), hl, st);
            if (e != cudaSuccess) return cuda_fail(e, "tessellation stage launch");
        }
    }
    return STENCIL_OK;
}

}  // namespace sg

using namespace sg;

// Host-only: counts[s * N + x] = the levels 1..levels at which stage s of one
// time tile updates point x (N = the product of the extents).  Returns
// STENCIL_ERR_INVALID_ARG when a segment is shorter than 2 levels radius.
extern "C" stencil_status_t stencil_tess_counts(int32_t dim, const int64_t *shape, int32_t radius, int32_t levels,
                                                int32_t tile, int32_t periodic, int32_t *counts) {
    if (dim < 1 || dim > 3 || !shape || radius < 1 || levels < 1 || tile < 1 || !counts) {
        set_error("invalid argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    int64_t N = 1;
    for (int a = 0; a < dim; ++a) {
        if (shape[a] < 1 || shape[a] > (1 << 20)) { set_error("extents 1..2^20"); return STENCIL_ERR_INVALID_ARG; }
        N *= shape[a];
    }
    if (N > (1ll << 26)) { set_error("at most 2^26 points"); return STENCIL_ERR_INVALID_ARG; }
    TessGeo g;
    if (!tess_geo(dim, shape, tile, levels, radius, periodic != 0, g)) {
        set_error("a segment is shorter than 2 levels radius");
        return STENCIL_ERR_INVALID_ARG;
    }
    std::fill(counts, counts + (dim + 1) * N, 0);
    const int n0 = g.ax[0].n, n1 = g.ax[1].n, n2 = g.ax[2].n;
    for (int s = 0; s <= dim; ++s) {
        tess_stage(g, s);
        for (int tile_i = 0; tile_i < g.tiles; ++tile_i) {
            int mask, idx[3];
            tess_tile(g, tile_i, mask, idx);
            for (int t = 1; t <= levels; ++t) {
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    if (a < 3 - dim) { lo[a] = 0; hi[a] = 1; }
                    else tess_range(g.ax[a], (mask >> (a - (3 - dim))) & 1, idx[a], t, radius, lo[a], hi[a]);
                }
                for (int i0 = lo[0]; i0 < hi[0]; ++i0)
                    for (int i1 = lo[1]; i1 < hi[1]; ++i1)
                        for (int i2 = lo[2]; i2 < hi[2]; ++i2) {
                            const int z = (i0 % n0 + n0) % n0, y = (i1 % n1 + n1) % n1, x = (i2 % n2 + n2) % n2;
                            counts[s * N + ((int64_t)z * n1 + y) * n2 + x] += 1;
                        }
            }
        }
    }
    return STENCIL_OK;
}
