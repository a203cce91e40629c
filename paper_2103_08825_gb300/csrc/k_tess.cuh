// k_tess.cuh -- tessellate tiling (paper Section 3.4, Fig. 6): T steps in
// time tiles of h levels, each time tile in d + 1 stages of concurrent tiles,
// with no redundant computation.
//
// One axis of extent n is cut at e_0 = 0 < e_1 < ... < e_m = n into segments
// of at least 2 h r points.  At level t (1 <= t <= h) of a time tile:
//   triangle i   updates [e_i + t r, e_{i+1} - t r)  (shrinking, Fig. 6a);
//   inverted j   updates [e_j - t r, e_j + t r)      (expanding, Fig. 6b),
//                around every cut -- on a periodic axis e_0 = e_m is one cut
//                and the range wraps; on a Dirichlet axis the two outer cuts
//                are clipped to the domain.
// For every t the triangles and inverted triangles partition the axis, so
// each point is updated once per level: after a triangle a point holds the
// level min(t_max) of Fig. 6's (0,1,..,h,..,1,0) profile, the inverted
// triangles add the complement (h,..,1,0,1,..,h), and every point ends at h.
// In d dimensions a tile is a product of per-axis ranges; stage s runs, all
// at once, the tiles with inverted ranges on exactly s axes (d + 1 stages, as
// the paper states).  A level-t update reads level t - 1 within r on every
// axis, which lies in the same tile (earlier level) or in a tile of an
// earlier stage, whose points are then at level t - 1 or t: the slope r of
// the tile sides keeps every point within one level of its neighbours, so two
// buffers by level parity hold all the values the stage reads.
//
// Kernel: one launch per stage, one CTA per tile (grid-stride), the levels of
// the tile in order with a CTA barrier between them; values are read from the
// parity buffer of level t - 1 and written to that of level t (global memory:
// a tile's working set stays in L1/L2).  Each point's sum is the plain
// kernel's (one multiply, then FMAs in lexicographic order), so results are
// bit-identical to stencil_run's.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

// An axis: cuts e_i = i * b for i < m, e_m = n (the last segment takes the
// remainder, b <= width < 2b; a single segment when n < 2b).
struct TessAxis {
    int n, b, m;
    int periodic;
};

__host__ __device__ __forceinline__ int tess_cut(const TessAxis &a, int i) { return i >= a.m ? a.n : i * a.b; }

// Number of tiles of a kind on an axis: m triangles; m inverted (periodic,
// e_0 = e_m) or m + 1 (Dirichlet).
__host__ __device__ __forceinline__ int tess_count(const TessAxis &a, bool inverted) {
    return inverted ? (a.periodic ? a.m : a.m + 1) : a.m;
}

// Range [lo, hi) (virtual coordinates: a periodic inverted range may start
// below 0) that tile i of the kind updates at level t; empty when lo >= hi.
__host__ __device__ __forceinline__ void tess_range(const TessAxis &a, bool inverted, int i, int t, int r, int &lo,
                                                    int &hi) {
    if (!inverted) {
        lo = tess_cut(a, i) + t * r;
        hi = tess_cut(a, i + 1) - t * r;
    } else {
        const int e = tess_cut(a, i);
        lo = e - t * r;
        hi = e + t * r;
        if (!a.periodic) {
            if (lo < 0) lo = 0;
            if (hi > a.n) hi = a.n;
        }
    }
}

// The levels t at which tile i of the kind updates coordinate c (virtual) of
// the axis: [lo, hi] (empty when lo > hi; hi open-ended for an expanding tile).
__host__ __device__ __forceinline__ void tess_levels(const TessAxis &a, bool inverted, int i, int c, int r, int &lo,
                                                     int &hi) {
    if (!inverted) {
        // c in [e_i + t r, e_{i+1} - t r)  <=>  t r <= min(c - e_i, e_{i+1} - 1 - c)
        const int m = min(c - tess_cut(a, i), tess_cut(a, i + 1) - 1 - c);
        lo = 1;
        hi = m < 0 ? 0 : m / r;
    } else {
        // c in [e - t r, e + t r)  <=>  t r >= e - c and t r > c - e
        const int e = tess_cut(a, i);
        lo = c >= e ? (c - e) / r + 1 : (e - c + r - 1) / r;
        hi = 1 << 30;
    }
}

struct TessGeo {
    int d;
    TessAxis ax[3];            // axis 0 outermost (padded to 3 with n = 1 axes)
    int h;                     // levels of the time tile
    int r;
    // tiles of a stage: combos of inverted axes (bit a set: axis a inverted)
    int ncombo;
    int combo[3];              // at most C(3, s) <= 3 combos per stage
    int combo_tiles[3];        // tiles of each combo
    int tiles;                 // tiles of the stage
};

// The stage's combos: every set of exactly s inverted axes among the d.
inline void tess_stage(TessGeo &g, int s) {
    g.ncombo = 0;
    g.tiles = 0;
    for (int mask = 0; mask < (1 << g.d); ++mask) {
        if (__builtin_popcount(mask) != s) continue;
        int n = 1;
        for (int a = 0; a < g.d; ++a) n *= tess_count(g.ax[3 - g.d + a], (mask >> a) & 1);
        g.combo[g.ncombo] = mask;
        g.combo_tiles[g.ncombo] = n;
        g.tiles += n;
        ++g.ncombo;
    }
}

// Tile `t` of the stage -> its inverted mask (over the d stencil axes, bit a
// = axis 3 - d + a) and its index on each of the 3 padded axes.
__host__ __device__ __forceinline__ void tess_tile(const TessGeo &g, int t, int &mask, int idx[3]) {
    int c = 0;
    while (c + 1 < g.ncombo && t >= g.combo_tiles[c]) {
        t -= g.combo_tiles[c];
        ++c;
    }
    mask = g.combo[c];
    idx[0] = idx[1] = idx[2] = 0;
    for (int a = g.d - 1; a >= 0; --a) {
        const int cnt = tess_count(g.ax[3 - g.d + a], (mask >> a) & 1);
        idx[3 - g.d + a] = t % cnt;
        t /= cnt;
    }
}

template <typename C> struct TessParams {
    GridGeom<C> g;
    void *buf[2];              // level parity buffers: level t lives in buf[t & 1]
    int t0;                    // global level at the start of the time tile
    int hlev;                  // levels of this time tile (<= h of the geometry)
    TessGeo geo;
    C w[kMaxPts];              // evaluation order
};

// One stage of one time tile: CTAs take its tiles (grid-stride) and advance
// each through levels 1..hlev in order.
template <int DT, int D, int R, int PAT>
__global__ void __launch_bounds__(256) tess_kernel(const __grid_constant__ TessParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using Sh = Shape<D, R, PAT>;
    const TessGeo &g = p.geo;
    const int n0 = g.ax[0].n, n1 = g.ax[1].n, n2 = g.ax[2].n;
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    const C bval = p.g.bval;
    for (int tile = blockIdx.x; tile < g.tiles; tile += gridDim.x) {
        int mask, idx[3];
        tess_tile(g, tile, mask, idx);
        for (int t = 1; t <= p.hlev; ++t) {
            const S *__restrict__ src = static_cast<const S *>(p.buf[(p.t0 + t - 1) & 1]);
            S *__restrict__ dst = static_cast<S *>(p.buf[(p.t0 + t) & 1]);
            int lo[3], hi[3];
            int ext = 1;   // points of the tile at this level (a tile is at most a few 10^4 points)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a < 3 - D) {
                    lo[a] = 0;
                    hi[a] = 1;
                } else {
                    tess_range(g.ax[a], (mask >> (a - (3 - D))) & 1, idx[a], t, R, lo[a], hi[a]);
                }
                ext *= hi[a] > lo[a] ? hi[a] - lo[a] : 0;
            }
            const int e1 = hi[1] - lo[1], e2 = hi[2] - lo[2];
            for (int q = threadIdx.x; q < ext; q += blockDim.x) {
                // 32-bit index arithmetic: a 64-bit division per point cost
                // more than the stencil itself
                const int qq = q / e2;
                int i2 = lo[2] + (q - qq * e2);
                const int q1 = qq / e1;
                int i1 = lo[1] + (qq - q1 * e1), i0 = lo[0] + q1;
                // virtual coordinates of a wrapping inverted range
                if (i0 < 0) i0 += n0; else if (i0 >= n0) i0 -= n0;
                if (i1 < 0) i1 += n1; else if (i1 >= n1) i1 -= n1;
                if (i2 < 0) i2 += n2; else if (i2 >= n2) i2 -= n2;
                C acc = C(0);
                bool first = true;
#pragma unroll
                for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz)
#pragma unroll
                    for (int oy = (D >= 2 ? -R : 0); oy <= (D >= 2 ? R : 0); ++oy)
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox) {
                            if (!Sh::inc(oz, oy, ox)) continue;
                            int z = i0 + oz, y = i1 + oy, x = i2 + ox;
                            bool ok = true;
                            if (z < 0 || z >= n0) { if (periodic) z = (int)wrap_idx(z, n0); else ok = false; }
                            if (y < 0 || y >= n1) { if (periodic) y = (int)wrap_idx(y, n1); else ok = false; }
                            if (x < 0 || x >= n2) { if (periodic) x = (int)wrap_idx(x, n2); else ok = false; }
                            const C v = ok ? to_c(src[((int64_t)z * n1 + y) * n2 + x]) : bval;
                            const C w = p.w[Sh::widx(oz, oy, ox)];
                            acc = first ? op_mul(w, v) : op_fma(w, v, acc);
                            first = false;
                        }
                dst[((int64_t)i0 * n1 + i1) * n2 + i2] = from_c<S>(acc);
            }
            __syncthreads();   // level t of the tile is complete before level t + 1 reads it
        }
    }
}

// The same stage with each tile's levels in shared memory: the tile loads
// both level-parity buffers over its region -- per axis the union of its
// ranges over the levels (the first level's range for a shrinking tile, the
// last one's for an expanding tile) plus r on every side -- once, advances
// levels 1..hlev there (each level read from the parity buffer of the level
// before), and writes both buffers back at the points it updated.  Every value
// a level reads is this tile's own earlier level or a value an earlier stage
// left in the parity buffers (as in tess_kernel); within a stage every point
// is updated by one tile only, and nothing else in the stage writes the
// buffers there, so the result is tess_kernel's, bit for bit.  The launcher uses it
// where the region fits in shared memory and does not wrap onto itself.
template <int DT, int D, int R, int PAT>
__global__ void __launch_bounds__(256) tess_smem_kernel(const __grid_constant__ TessParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using Sh = Shape<D, R, PAT>;
    extern __shared__ __align__(16) unsigned char tsm[];
    const TessGeo &g = p.geo;
    const int n[3] = {g.ax[0].n, g.ax[1].n, g.ax[2].n};
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    const C bval = p.g.bval;
    S *const gb0 = static_cast<S *>(p.buf[0]);
    S *const gb1 = static_cast<S *>(p.buf[1]);
    for (int tile = blockIdx.x; tile < g.tiles; tile += gridDim.x) {
        int mask, idx[3];
        tess_tile(g, tile, mask, idx);
        int ulo[3], uhi[3], elo[3], ext[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a < 3 - D) {
                ulo[a] = 0;
                uhi[a] = 1;
                elo[a] = 0;
                ext[a] = 1;
            } else {
                const bool inv = (mask >> (a - (3 - D))) & 1;
                tess_range(g.ax[a], inv, idx[a], inv ? p.hlev : 1, R, ulo[a], uhi[a]);
                elo[a] = ulo[a] - R;
                ext[a] = uhi[a] - ulo[a] + 2 * R;
            }
        }
        const int ne = ext[0] * ext[1] * ext[2];
        S *const s0 = reinterpret_cast<S *>(tsm);
        S *const s1 = s0 + ne;
        // physical index of virtual (z, y, x), or -1 outside a Dirichlet domain
        auto phys = [&](int z, int y, int x) -> int64_t {
            if (z < 0 || z >= n[0]) { if (!periodic) return -1; z = (int)wrap_idx(z, n[0]); }
            if (y < 0 || y >= n[1]) { if (!periodic) return -1; y = (int)wrap_idx(y, n[1]); }
            if (x < 0 || x >= n[2]) { if (!periodic) return -1; x = (int)wrap_idx(x, n[2]); }
            return ((int64_t)z * n[1] + y) * n[2] + x;
        };
        for (int q = threadIdx.x; q < ne; q += blockDim.x) {
            const int q1 = q / ext[2], q0 = q1 / ext[1];
            const int64_t i = phys(elo[0] + q0, elo[1] + (q1 - q0 * ext[1]), elo[2] + (q - q1 * ext[2]));
            s0[q] = i >= 0 ? gb0[i] : from_c<S>(bval);
            s1[q] = i >= 0 ? gb1[i] : from_c<S>(bval);
        }
        __syncthreads();
        for (int t = 1; t <= p.hlev; ++t) {
            const S *src = ((p.t0 + t - 1) & 1) ? s1 : s0;
            S *dst = ((p.t0 + t) & 1) ? s1 : s0;
            int lo[3], hi[3];
            int cnt = 1;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a < 3 - D) {
                    lo[a] = 0;
                    hi[a] = 1;
                } else {
                    tess_range(g.ax[a], (mask >> (a - (3 - D))) & 1, idx[a], t, R, lo[a], hi[a]);
                }
                cnt *= hi[a] > lo[a] ? hi[a] - lo[a] : 0;
            }
            const int e1 = hi[1] - lo[1], e2 = hi[2] - lo[2];
            for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
                const int qq = q / e2;
                const int q1 = qq / e1;
                // shared-memory coordinates of the point
                const int c0 = lo[0] + q1 - elo[0], c1 = lo[1] + (qq - q1 * e1) - elo[1],
                          c2 = lo[2] + (q - qq * e2) - elo[2];
                C acc = C(0);
                bool first = true;
#pragma unroll
                for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz)
#pragma unroll
                    for (int oy = (D >= 2 ? -R : 0); oy <= (D >= 2 ? R : 0); ++oy)
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox) {
                            if (!Sh::inc(oz, oy, ox)) continue;
                            const C v = to_c(src[((c0 + oz) * ext[1] + (c1 + oy)) * ext[2] + (c2 + ox)]);
                            const C w = p.w[Sh::widx(oz, oy, ox)];
                            acc = first ? op_mul(w, v) : op_fma(w, v, acc);
                            first = false;
                        }
                dst[(c0 * ext[1] + c1) * ext[2] + c2] = from_c<S>(acc);
            }
            __syncthreads();
        }
        // both parity buffers back at the points this tile updated at some
        // level (the product of its per-axis unions also holds points that
        // another tile of the same stage, inverted on another axis, updates)
        const int u1 = uhi[1] - ulo[1], u2 = uhi[2] - ulo[2];
        const int nu = (uhi[0] - ulo[0]) * u1 * u2;
        for (int q = threadIdx.x; q < nu; q += blockDim.x) {
            const int qq = q / u2, q0 = qq / u1;
            const int z = ulo[0] + q0, y = ulo[1] + (qq - q0 * u1), x = ulo[2] + (q - qq * u2);
            const int c3[3] = {z, y, x};
            int tlo = 1, thi = p.hlev;
#pragma unroll
            for (int a = 3 - D; a < 3; ++a) {
                int lo, hi;
                tess_levels(g.ax[a], (mask >> (a - (3 - D))) & 1, idx[a], c3[a], R, lo, hi);
                tlo = max(tlo, lo);
                thi = min(thi, hi);
            }
            if (tlo > thi) continue;   // not one of this tile's points at any level
            const int64_t i = phys(z, y, x);
            if (i < 0) continue;
            const int c = ((z - elo[0]) * ext[1] + (y - elo[1])) * ext[2] + (x - elo[2]);
            gb0[i] = s0[c];
            gb1[i] = s1[c];
        }
        __syncthreads();   // the next tile reuses the shared memory
    }
}

// Shared memory the smem kernel needs for geometry g (0: it does not apply --
// a region larger than the budget, or wrapping onto itself on a periodic axis)
inline size_t tess_smem_bytes(const TessGeo &g, int r, size_t elem) {
    size_t pts = 1;
    for (int a = 0; a < 3; ++a) {
        const TessAxis &x = g.ax[a];
        if (x.n == 1 && x.b == 1) continue;   // padded axis
        const int seg = x.m <= 1 ? x.n : std::max(x.b, x.n - (x.m - 1) * x.b);
        const int inv = 2 * g.h * r + 2 * r;
        if (x.periodic && inv > x.n) return 0;
        pts *= (size_t)std::max(seg, inv);
    }
    const size_t bytes = 2 * pts * elem;
    return bytes <= 160 * 1024 ? bytes : 0;
}

template <int DT, int D, int R, int PAT>
cudaError_t launch_tess_t(const stencil_plan_s &P, const TessGeo &geo, void *b0, void *b1, int t0, int hlev,
                          cudaStream_t st) {
    using C = typename Traits<DT>::C;
    TessParams<C> p;
    p.g.n0 = P.n[0];
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.buf[0] = b0;
    p.buf[1] = b1;
    p.t0 = t0;
    p.hlev = hlev;
    p.geo = geo;
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    int64_t grid = geo.tiles;
    if (grid < 1) return cudaSuccess;
    const size_t smem = tess_smem_bytes(geo, R, sizeof(typename Traits<DT>::S));
    if (smem > 0) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(tess_smem_kernel<DT, D, R, PAT>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        int bps = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tess_smem_kernel<DT, D, R, PAT>, 256,
                                                                      smem);
        if (e != cudaSuccess) return e;
        grid = std::min<int64_t>(grid, (int64_t)P.sm_count * std::max(bps, 1));
        tess_smem_kernel<DT, D, R, PAT><<<(unsigned)grid, 256, smem, st>>>(p);
        return cudaGetLastError();
    }
    if (grid > (int64_t)P.sm_count * 8) grid = (int64_t)P.sm_count * 8;
    tess_kernel<DT, D, R, PAT><<<(unsigned)grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

template <int DT, int D>
cudaError_t launch_tess_d(const stencil_plan_s &P, const TessGeo &geo, void *b0, void *b1, int t0, int hlev,
                          cudaStream_t st) {
    const bool box = P.pattern == STENCIL_BOX;
    switch (P.r) {
        case 1: return box ? launch_tess_t<DT, D, 1, STENCIL_BOX>(P, geo, b0, b1, t0, hlev, st)
                           : launch_tess_t<DT, D, 1, STENCIL_STAR>(P, geo, b0, b1, t0, hlev, st);
        case 2: return box ? launch_tess_t<DT, D, 2, STENCIL_BOX>(P, geo, b0, b1, t0, hlev, st)
                           : launch_tess_t<DT, D, 2, STENCIL_STAR>(P, geo, b0, b1, t0, hlev, st);
        case 3: return box ? launch_tess_t<DT, D, 3, STENCIL_BOX>(P, geo, b0, b1, t0, hlev, st)
                           : launch_tess_t<DT, D, 3, STENCIL_STAR>(P, geo, b0, b1, t0, hlev, st);
    }
    return cudaErrorInvalidValue;
}

template <int DT>
cudaError_t launch_tess_dt(const stencil_plan_s &P, const TessGeo &geo, void *b0, void *b1, int t0, int hlev,
                           cudaStream_t st) {
    switch (P.dim) {
        case 1: return launch_tess_d<DT, 1>(P, geo, b0, b1, t0, hlev, st);
        case 2: return launch_tess_d<DT, 2>(P, geo, b0, b1, t0, hlev, st);
        case 3: return launch_tess_d<DT, 3>(P, geo, b0, b1, t0, hlev, st);
    }
    return cudaErrorInvalidValue;
}

#define SG_DECL_TESS(DT)                                                                                   \
    cudaError_t launch_tess_##DT(const stencil_plan_s &, const TessGeo &, void *, void *, int, int, cudaStream_t);
SG_DECL_TESS(F32)
SG_DECL_TESS(F64)
SG_DECL_TESS(BF16)
SG_DECL_TESS(F16)
SG_DECL_TESS(I32)
#undef SG_DECL_TESS

}  // namespace sg
