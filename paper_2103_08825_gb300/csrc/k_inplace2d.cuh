// k_inplace2d.cuh -- 2D Jacobi sweep advanced in place: one grid plus the
// border rings of its tiles, instead of two grids.
//
// The paper's in-place update (Section 3.3, last paragraph): with the time
// loop unrolled by k = 2, input and output of a pass sit at even time levels,
// so a single array suffices -- the sequential sweep keeps every old value it
// still needs in registers ("vrl") before overwriting it.  On a GPU the tiles
// of a pass run concurrently, and a tile's overlapped window reads its
// neighbours' cells, which they overwrite during the same pass.  So each tile
// also keeps a copy of its "ring" -- the cells within H columns or rK rows of
// its border, the only cells any neighbour's window reaches -- in a small
// side buffer: a pass reads its own cells from the grid (each row before the
// tile overwrites it: stores trail loads by rK rows) and its neighbours' cells
// from the rings of the pass before, and writes its new values to the grid
// and its new ring to the other side buffer.  The side buffers take about
// 2 (2 rK / Ly + 2 H / BW) of a grid, so the sweep needs about half the
// memory of the two-grid form.  Any k works, not only 2.
//
// Tiles: column bands of BW = W - 2H columns (H >= rK, 16-byte aligned, fixed
// for all passes from the plan's k) and row chunks of Ly rows.  One warp per
// job, one launch per pass, loads through registers (as the fused kernel's
// PROD_REG path); the update order is the fused kernel's, so results are
// bit-identical to stencil_run's.
#pragma once

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

struct InplGeo {
    int nx, ny;
    int BW, H;      // band width and x halo (window = BW + 2H <= 32 V columns)
    int Ly, rK;     // chunk height and the rows of ring kept at each end (R k of the plan)
    int bands, chunks;
    int ring;       // elements of one tile's ring: 2 rK BW + 2 Ly H
};

template <typename C> struct InplParams {
    GridGeom<C> g;          // n1 = ny, n2 = nx
    void *u;                // the grid, advanced in place
    const void *ring_in;    // rings after the previous pass
    void *ring_out;         // rings after this pass
    InplGeo t;
    int vec_ok;
    JobCtl *ctl;            // job tickets (left at zero by the launch's last warp)
    long long jobs;
    C w[49];                // evaluation order; up to the r = 3 box
};

// Position of in-domain cell (x, y) in its owning tile's ring: the top rows,
// bottom rows, left columns, right columns, in that order of preference.  A
// cell outside every strip (reached only through a periodic window that wraps
// onto itself, beyond every stored output's dependency cone) maps to the
// ring's first element: in bounds, and never used for a stored result.
__host__ __device__ __forceinline__ int64_t ring_index(const InplGeo &t, int x, int y) {
    const int b = x / t.BW, c = y / t.Ly;
    const int rx = x - b * t.BW, ry = y - c * t.Ly;
    const int bw = t.nx - b * t.BW < t.BW ? t.nx - b * t.BW : t.BW;
    const int ly = t.ny - c * t.Ly < t.Ly ? t.ny - c * t.Ly : t.Ly;
    const int tr = t.rK < ly ? t.rK : ly, tc = t.H < bw ? t.H : bw;
    const int64_t base = ((int64_t)c * t.bands + b) * t.ring;
    if (ry < tr) return base + (int64_t)ry * t.BW + rx;
    if (ry >= ly - tr) return base + (int64_t)t.rK * t.BW + (int64_t)(ry - (ly - tr)) * t.BW + rx;
    if (rx < tc) return base + 2ll * t.rK * t.BW + (int64_t)ry * t.H + rx;
    if (rx >= bw - tc) return base + 2ll * t.rK * t.BW + (int64_t)t.Ly * t.H + (int64_t)ry * t.H + (rx - (bw - tc));
    return base;
}

// Record the new value of own cell (rx, ry) of tile (b, c) in every strip of
// its ring that holds it.
template <typename S>
__device__ __forceinline__ void ring_put(const InplGeo &t, S *ring, int b, int c, int bw, int ly, int rx, int ry,
                                         S val) {
    const int tr = t.rK < ly ? t.rK : ly, tc = t.H < bw ? t.H : bw;
    S *base = ring + ((int64_t)c * t.bands + b) * t.ring;
    if (ry < tr) base[(int64_t)ry * t.BW + rx] = val;
    if (ry >= ly - tr) base[(int64_t)t.rK * t.BW + (int64_t)(ry - (ly - tr)) * t.BW + rx] = val;
    if (rx < tc) base[2ll * t.rK * t.BW + (int64_t)ry * t.H + rx] = val;
    if (rx >= bw - tc) base[2ll * t.rK * t.BW + (int64_t)t.Ly * t.H + (int64_t)ry * t.H + (rx - (bw - tc))] = val;
}

// Fill the rings from the grid (before the first pass).
template <typename S>
__global__ void __launch_bounds__(256) inplace_ring_init(const S *__restrict__ u, S *__restrict__ ring, InplGeo t) {
    const int64_t total = (int64_t)t.bands * t.chunks * t.ring;
    for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < total; i += (int64_t)gridDim.x * 256) {
        const int tile = (int)(i / t.ring), e = (int)(i - (int64_t)tile * t.ring);
        const int b = tile % t.bands, c = tile / t.bands;
        const int bw = t.nx - b * t.BW < t.BW ? t.nx - b * t.BW : t.BW;
        const int ly = t.ny - c * t.Ly < t.Ly ? t.ny - c * t.Ly : t.Ly;
        const int tr = t.rK < ly ? t.rK : ly, tc = t.H < bw ? t.H : bw;
        int rx, ry;
        bool ok;
        if (e < t.rK * t.BW) {
            ry = e / t.BW; rx = e % t.BW; ok = ry < tr && rx < bw;
        } else if (e < 2 * t.rK * t.BW) {
            const int q = e - t.rK * t.BW;
            ry = ly - tr + q / t.BW; rx = q % t.BW; ok = q / t.BW < tr && rx < bw;
        } else if (e < 2 * t.rK * t.BW + t.Ly * t.H) {
            const int q = e - 2 * t.rK * t.BW;
            ry = q / t.H; rx = q % t.H; ok = ry < ly && rx < tc;
        } else {
            const int q = e - 2 * t.rK * t.BW - t.Ly * t.H;
            ry = q / t.H; rx = bw - tc + q % t.H; ok = ry < ly && q % t.H < tc;
        }
        if (ok) ring[i] = u[(int64_t)(c * t.Ly + ry) * t.nx + b * t.BW + rx];
    }
}

// V values of virtual row yv at columns xl .. xl + V - 1 for the tile with
// output [xo0, xo0 + bw) x [yo0, yo1): the tile's own cells from the grid,
// other cells from the rings of the previous pass, cells outside a Dirichlet
// domain the boundary value, a periodic grid wrapped.
template <int DT>
__device__ __forceinline__ void inpl_load(const InplParams<typename Traits<DT>::C> &p,
                                          const typename Traits<DT>::S *__restrict__ u,
                                          const typename Traits<DT>::S *__restrict__ ring, int yv, int xl, int xo0,
                                          int bw, int yo0, int yo1, typename Traits<DT>::C *out) {
    constexpr int V = Traits<DT>::V;
    const int nx = p.t.nx, ny = p.t.ny;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    const typename Traits<DT>::C bval = p.g.bval;
    int y = yv;
    if (y < 0 || y >= ny) {
        if (dir) {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = bval;
            return;
        }
        y = (int)wrap_idx(y, ny);
    }
    const bool own_row = yv >= yo0 && yv < yo1;
    // the grid is read through L2 (ld.global.cg): other tiles write it during
    // the launch, and its cache lines straddle tile borders
    if (own_row && p.vec_ok && xl >= xo0 && xl + V <= xo0 + bw) {
        ldvec<DT, true>(u + (int64_t)y * nx + xl, out);
        return;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int xv = xl + v;
        int x = xv;
        if (x < 0 || x >= nx) {
            if (dir) { out[v] = bval; continue; }
            x = (int)wrap_idx(x, nx);
        }
        if (own_row && xv >= xo0 && xv < xo0 + bw) out[v] = to_c(__ldcg(u + (int64_t)y * nx + xv));
        else out[v] = to_c(ring[ring_index(p.t, x, y)]);
    }
}

// One job: tile (b, c) advanced K steps in place.  The level loop is the
// fused kernel's (fused2d_job), with the window start and output columns set
// by the ring geometry at run time.
template <int DT, int R, int PAT, int K, bool MASK>
__device__ __forceinline__ void inplace2d_job(const InplParams<typename Traits<DT>::C> &p, int b, int c, int lane) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using Sh = Shape<2, R, PAT>;
    constexpr int V = Traits<DT>::V, NS = 2 * R;
    constexpr int U = lcm_c(NS, F2_PREF);
    constexpr uint32_t FULLM = (1u << V) - 1u;
    S *__restrict__ u = static_cast<S *>(p.u);
    const S *__restrict__ ring = static_cast<const S *>(p.ring_in);
    S *__restrict__ ring_out = static_cast<S *>(p.ring_out);
    const C *wr = p.w;
    const C bval = p.g.bval;
    const int nx = p.t.nx, ny = p.t.ny;
    const int xo0 = b * p.t.BW, bw = nx - xo0 < p.t.BW ? nx - xo0 : p.t.BW;
    const int yo0 = c * p.t.Ly, yo1 = yo0 + p.t.Ly < ny ? yo0 + p.t.Ly : ny;
    const int xl = xo0 - p.t.H + lane * V;
    const int yi0 = yo0 - R * K;
    const int nsteps = (yo1 - yo0) + 2 * R * K;
    const int nsp = round_up_c(nsteps, U);
    uint32_t cmask = 0;
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (xl + v >= 0 && xl + v < nx) cmask |= 1u << v;
    const bool need_cmask = MASK && __any_sync(0xffffffffu, cmask != FULLM);
    bool keep[V];
#pragma unroll
    for (int v = 0; v < V; ++v) keep[v] = (cmask >> v) & 1u;

    C pre[F2_PREF][V];
#pragma unroll
    for (int q = 0; q < F2_PREF; ++q) inpl_load<DT>(p, u, ring, yi0 + q, xl, xo0, bw, yo0, yo1, pre[q]);
    C P[K][NS][V];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int m = 0; m < NS; ++m)
#pragma unroll
            for (int v = 0; v < V; ++v) P[s][m][v] = C(0);
    for (int i0 = 0; i0 < nsp; i0 += U) {
#pragma unroll
        for (int ph = 0; ph < U; ++ph) {
            const int yin = yi0 + i0 + ph;
            C cur[V];
#pragma unroll
            for (int v = 0; v < V; ++v) cur[v] = pre[ph % F2_PREF][v];
            // rows are read F2_PREF ahead of the row entering level 0 and
            // written K R rows behind it: a row of the tile is never read
            // after the tile has overwritten it
            inpl_load<DT>(p, u, ring, yin + F2_PREF, xl, xo0, bw, yo0, yo1, pre[ph % F2_PREF]);
            if constexpr (MASK) {
                if ((unsigned)yin >= (unsigned)ny) {
#pragma unroll
                    for (int v = 0; v < V; ++v) cur[v] = bval;
                } else if (need_cmask) {
#pragma unroll
                    for (int v = 0; v < V; ++v) cur[v] = keep[v] ? cur[v] : bval;
                }
            }
#pragma unroll
            for (int s = 0; s < K; ++s) {
                C ext[V + 2 * R];
#pragma unroll
                for (int v = 0; v < V; ++v) ext[R + v] = cur[v];
#pragma unroll
                for (int qq = 0; qq < R; ++qq) {
                    ext[R - 1 - qq] = __shfl_up_sync(0xffffffffu, cur[V - 1 - qq % V], qq / V + 1);
                    ext[R + V + qq] = __shfl_down_sync(0xffffffffu, cur[qq % V], qq / V + 1);
                }
                C emit[V];
                const int s0 = ph % NS;
#pragma unroll
                for (int v = 0; v < V; ++v) emit[v] = P[s][s0][v];
#pragma unroll
                for (int ox = -R; ox <= R; ++ox)
                    if (Sh::inc(0, R, ox)) row_fma_s<C, V>(wr[Sh::widx(0, R, ox)], &ext[R + ox], emit);
#pragma unroll
                for (int m = 1; m < NS; ++m) {
                    const int oy = R - m, sl = (ph + m) % NS;
#pragma unroll
                    for (int ox = -R; ox <= R; ++ox)
                        if (Sh::inc(0, oy, ox)) row_fma_s<C, V>(wr[Sh::widx(0, oy, ox)], &ext[R + ox], P[s][sl]);
                }
                {
                    bool first = true;
#pragma unroll
                    for (int ox = -R; ox <= R; ++ox) {
                        if (!Sh::inc(0, -R, ox)) continue;
                        if (first) row_mul_s<C, V>(wr[Sh::widx(0, -R, ox)], &ext[R + ox], P[s][s0]);
                        else row_fma_s<C, V>(wr[Sh::widx(0, -R, ox)], &ext[R + ox], P[s][s0]);
                        first = false;
                    }
                }
                if constexpr (MASK) {
                    const int ye = yin - (s + 1) * R;
                    if ((unsigned)ye >= (unsigned)ny) {
#pragma unroll
                        for (int v = 0; v < V; ++v) emit[v] = bval;
                    } else if (need_cmask) {
#pragma unroll
                        for (int v = 0; v < V; ++v) emit[v] = keep[v] ? emit[v] : bval;
                    }
                }
#pragma unroll
                for (int v = 0; v < V; ++v) cur[v] = emit[v];
            }
            // level K: the tile's own cells, to the grid and to the new ring
            const int yout = yin - K * R;
            if (yout >= yo0 && yout < yo1) {
                S *rowp = u + (int64_t)yout * nx;
                if (p.vec_ok && xl >= xo0 && xl + V <= xo0 + bw) {
                    stvec<DT>(rowp + xl, cur);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (xl + v >= xo0 && xl + v < xo0 + bw) rowp[xl + v] = from_c<S>(cur[v]);
                }
                const int ry = yout - yo0, ly = yo1 - yo0;
                const int tr = p.t.rK < ly ? p.t.rK : ly, tc = p.t.H < bw ? p.t.H : bw;
                const int rx0 = xl - xo0;
                // ring cells: the first / last rK rows, or the first / last H columns
                if (ry < tr || ry >= ly - tr || rx0 < tc || rx0 + V > bw - tc) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (rx0 + v >= 0 && rx0 + v < bw)
                            ring_put<S>(p.t, ring_out, b, c, bw, ly, rx0 + v, ry, from_c<S>(cur[v]));
                }
            }
        }
    }
}

template <int DT, int R, int PAT, int K>
__global__ void __launch_bounds__(F2_NW * 32) inplace2d_kernel(const __grid_constant__ InplParams<typename Traits<DT>::C> p) {
    const int lane = threadIdx.x & 31;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    const int W = 32 * Traits<DT>::V;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&p.ctl->ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)p.jobs) break;
        const int b = (int)(t % (unsigned)p.t.bands), c = (int)(t / (unsigned)p.t.bands);
        const int xw0 = b * p.t.BW - p.t.H, yo0 = c * p.t.Ly;
        const int yo1 = yo0 + p.t.Ly < p.t.ny ? yo0 + p.t.Ly : p.t.ny;
        // a window inside the domain never meets a Dirichlet cell
        const bool interior = !dir || (xw0 >= 0 && xw0 + W <= p.t.nx && yo0 - R * K >= 0 && yo1 + R * K <= p.t.ny);
        if (interior) inplace2d_job<DT, R, PAT, K, false>(p, b, c, lane);
        else inplace2d_job<DT, R, PAT, K, true>(p, b, c, lane);
    }
    __syncwarp();
    if (lane == 0 && worker_exit_is_last(&p.ctl->exited, gridDim.x * F2_NW)) {
        p.ctl->ticket = 0ull;
        p.ctl->exited = 0u;
    }
}

constexpr int INPL_KMAX = 4;   // fusion depths of the in-place sweep (radius 1)
// radius 2 fuses up to 2 steps, radius 3 one (the ring's halo grows with r k)
__host__ __device__ constexpr int inpl_kmax(int r) { return r == 1 ? INPL_KMAX : r == 2 ? 2 : 1; }

// Ring geometry for fusion depth k: bands and halo from k (kept for every
// pass, the last one included), chunks of about two jobs per resident warp.
inline InplGeo inpl_geo(const stencil_plan_s &P, int k) {
    InplGeo t;
    const int v = P.dtype == STENCIL_F64 ? 2 : 4;
    const int al = std::max(16 / (int)dtype_size(P.dtype), v);
    t.nx = (int)P.n[2];
    t.ny = (int)P.n[1];
    t.rK = P.r * k;
    t.H = (t.rK + al - 1) / al * al;
    t.BW = 32 * v - 2 * t.H;
    t.bands = (t.nx + t.BW - 1) / t.BW;
    const int64_t slots = (int64_t)P.sm_count * 16;
    int64_t chunks = std::max<int64_t>(1, 2 * slots / t.bands);
    int ly = (int)((t.ny + chunks - 1) / chunks);
    ly = std::max(ly, std::max(16, 2 * t.rK));
    t.Ly = std::min(ly, t.ny);
    t.chunks = (t.ny + t.Ly - 1) / t.Ly;
    t.ring = 2 * t.rK * t.BW + 2 * t.Ly * t.H;
    return t;
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_inpl_t(const stencil_plan_s &P, void *u, const void *ring_in, void *ring_out, const InplGeo &t,
                          cudaStream_t st) {
    using C = typename Traits<DT>::C;
    InplParams<C> p;
    if (P.np > (int)(sizeof(p.w) / sizeof(p.w[0]))) return cudaErrorInvalidValue;
    p.g.n0 = 1;
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.u = u;
    p.ring_in = ring_in;
    p.ring_out = ring_out;
    p.t = t;
    p.vec_ok = (P.n[2] % Traits<DT>::V == 0) && ((uintptr_t)u % 16 == 0);
    p.ctl = static_cast<JobCtl *>(P.d_ctr);
    p.jobs = (long long)t.bands * t.chunks;
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, inplace2d_kernel<DT, R, PAT, K>, F2_NW * 32, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = (p.jobs + F2_NW - 1) / F2_NW;
    const int64_t cap = (int64_t)P.sm_count * std::max(bps, 1);
    if (grid > cap) grid = cap;
    inplace2d_kernel<DT, R, PAT, K><<<(unsigned)grid, F2_NW * 32, 0, st>>>(p);
    return cudaGetLastError();
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_inpl_kr(const stencil_plan_s &P, int k, void *u, const void *ri, void *ro, const InplGeo &t,
                           cudaStream_t st) {
    if constexpr (K > inpl_kmax(R)) {
        return cudaErrorInvalidValue;
    } else {
        if (k == K) return launch_inpl_t<DT, R, PAT, K>(P, u, ri, ro, t, st);
        return launch_inpl_kr<DT, R, PAT, K + 1>(P, k, u, ri, ro, t, st);
    }
}

template <int DT>
cudaError_t launch_inpl_dt(const stencil_plan_s &P, int k, void *u, const void *ri, void *ro, const InplGeo &t,
                           cudaStream_t st) {
    const bool box = P.pattern == STENCIL_BOX;
    switch (P.r) {
        case 1: return box ? launch_inpl_kr<DT, 1, STENCIL_BOX, 1>(P, k, u, ri, ro, t, st)
                           : launch_inpl_kr<DT, 1, STENCIL_STAR, 1>(P, k, u, ri, ro, t, st);
        case 2: return box ? launch_inpl_kr<DT, 2, STENCIL_BOX, 1>(P, k, u, ri, ro, t, st)
                           : launch_inpl_kr<DT, 2, STENCIL_STAR, 1>(P, k, u, ri, ro, t, st);
        case 3: return box ? launch_inpl_kr<DT, 3, STENCIL_BOX, 1>(P, k, u, ri, ro, t, st)
                           : launch_inpl_kr<DT, 3, STENCIL_STAR, 1>(P, k, u, ri, ro, t, st);
    }
    return cudaErrorInvalidValue;
}

template <int DT>
cudaError_t launch_inpl_init_dt(const void *u, void *ring, const InplGeo &t, int sm_count, cudaStream_t st) {
    using S = typename Traits<DT>::S;
    const int64_t total = (int64_t)t.bands * t.chunks * t.ring;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)sm_count * 8) blocks = (int64_t)sm_count * 8;
    if (blocks < 1) blocks = 1;
    inplace_ring_init<S><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const S *>(u), static_cast<S *>(ring), t);
    return cudaGetLastError();
}

// one translation unit per storage type (k_inplace2d_<dtype>.cu)
#define SG_DECL_INPL(DT)                                                                                      \
    cudaError_t launch_inpl_##DT(const stencil_plan_s &, int, void *, const void *, void *, const InplGeo &,  \
                                 cudaStream_t);                                                             \
    cudaError_t launch_inpl_init_##DT(const void *, void *, const InplGeo &, int, cudaStream_t);
SG_DECL_INPL(F32)
SG_DECL_INPL(F64)
SG_DECL_INPL(BF16)
SG_DECL_INPL(F16)
SG_DECL_INPL(I32)
#undef SG_DECL_INPL

}  // namespace sg
