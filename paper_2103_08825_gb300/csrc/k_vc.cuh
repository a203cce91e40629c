// k_vc.cuh -- variable-coefficient sweeps: u_{t+1}[x] = sum_o c_o[x] u_t(x+o),
// a coefficient per offset and per grid point (the paper's Section 1 sweep
// with its weights made fields; not in the paper).  The coefficient field is
// stored offset-major in compact order, c[j N + x], in the arithmetic type
// (FP32 for F32 plans, FP64 for F64, uint32 bits for I32).
//
//   vc_plain_kernel   one step per launch, d = 1, 2, 3: a thread computes 4
//                     consecutive points of a row, reads their neighbours and
//                     their np coefficient vectors (offsets from a table);
//   vc2d_kernel       2D, K steps per pass: the fused kernel's warp-streamed
//                     partial rows (Section 3.3's unroll-and-jam), each term
//                     weighted by its target row's coefficient; coefficients
//                     are time-invariant, so one pass reads u once, writes it
//                     once and reads the np coefficient planes once from HBM
//                     (later levels find them in L1/L2): (2 + np) s bytes per
//                     point per pass, against (2 + np) s per step unfused.
// The order of the terms is the constant-weight kernels' (lexicographic
// offsets, one multiply then FMAs), so a constant field reproduces
// stencil_run bit for bit and every K gives the same result.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

template <typename C> struct VcParams {
    GridGeom<C> g;
    const void *src;
    void *dst;
    const C *coef;          // [np][N], compact order
    int64_t N;
    int vec_ok;             // rows, grids and coefficient planes allow V-wide access
    int np;                 // offsets
    short ci[kMaxPts];      // compact index of the j-th offset in evaluation order
    signed char off[kMaxPts][3];   // the j-th offset (one-step kernel), padded to 3D
    // fused 2D only
    int64_t jobs, bands, Ly;
    JobCtl *ctl;
};

// ------------------------------------------------------------ one step
// Offsets are taken from the parameter block at run time (one kernel per
// storage type for every dimension, radius and pattern).
template <int DT>
__global__ void __launch_bounds__(256) vc_plain_kernel(const __grid_constant__ VcParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    constexpr int VX = 4;
    const S *__restrict__ src = static_cast<const S *>(p.src);
    S *__restrict__ dst = static_cast<S *>(p.dst);
    const int64_t n0 = p.g.n0, n1 = p.g.n1, n2 = p.g.n2;
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    const C bval = p.g.bval;
    const int64_t groups = (n2 + VX - 1) / VX;
    const int64_t items = n0 * n1 * groups;
    for (int64_t it = blockIdx.x * 256ll + threadIdx.x; it < items; it += (int64_t)gridDim.x * 256) {
        const int64_t g = it % groups, row = it / groups;
        const int64_t i1 = row % n1, i0 = row / n1;
        const int64_t x0 = g * VX;
        const int64_t xbase = (i0 * n1 + i1) * n2;
        C acc[VX];
#pragma unroll 1
        for (int j = 0; j < p.np; ++j) {
            int64_t r0 = i0 + p.off[j][0], r1 = i1 + p.off[j][1];
            bool row_ok = true;
            if (r0 < 0 || r0 >= n0) { if (periodic) r0 = wrap_idx(r0, n0); else row_ok = false; }
            if (r1 < 0 || r1 >= n1) { if (periodic) r1 = wrap_idx(r1, n1); else row_ok = false; }
            const S *rowp = src + (r0 * n1 + r1) * n2;
            const C *cp = p.coef + (int64_t)p.ci[j] * p.N + xbase;
#pragma unroll
            for (int v = 0; v < VX; ++v) {
                if (x0 + v >= n2) continue;
                const int64_t x = x0 + v + p.off[j][2];
                C val;
                if (!row_ok) val = bval;
                else if (x >= 0 && x < n2) val = to_c(__ldg(rowp + x));
                else if (periodic) val = to_c(__ldg(rowp + wrap_idx(x, n2)));
                else val = bval;
                const C c = __ldg(cp + x0 + v);
                acc[v] = j == 0 ? op_mul(c, val) : op_fma(c, val, acc[v]);
            }
        }
#pragma unroll
        for (int v = 0; v < VX; ++v)
            if (x0 + v < n2) dst[xbase + x0 + v] = from_c<S>(acc[v]);
    }
}

// ------------------------------------------------------- fused 2D, K steps
// V coefficients of compact plane `cj` at (virtual) row y, columns xl..: in
// the domain read through the read-only path, wrapped on a periodic grid,
// zero outside a Dirichlet domain (those cells are reset to the boundary
// value anyway).
template <int DT>
__device__ __forceinline__ void vc_coef(const VcParams<typename Traits<DT>::C> &p, int cj, int y, int xl,
                                        typename Traits<DT>::C *out) {
    using C = typename Traits<DT>::C;
    constexpr int V = Traits<DT>::V;
    const int nx = (int)p.g.n2, ny = (int)p.g.n1;
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    if (y < 0 || y >= ny) {
        if (!periodic) {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = C(0);
            return;
        }
        y = (int)wrap_idx(y, ny);
    }
    const C *row = p.coef + (int64_t)cj * p.N + (int64_t)y * nx;
    if (p.vec_ok && xl >= 0 && xl + V <= nx) {
        if constexpr (sizeof(C) * V == 16) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(row + xl));
            const C *e = reinterpret_cast<const C *>(&q);
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = e[v];
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = __ldg(row + xl + v);
        }
        return;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        int x = xl + v;
        if (x < 0 || x >= nx) {
            if (!periodic) { out[v] = C(0); continue; }
            x = (int)wrap_idx(x, nx);
        }
        out[v] = __ldg(row + x);
    }
}

// acc[v] (+)= c[v] * x[v]
template <typename C, int V, bool FIRST>
__device__ __forceinline__ void vc_term(const C *c, const C *x, C *acc) {
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = FIRST ? op_mul(c[v], x[v]) : op_fma(c[v], x[v], acc[v]);
}

// One job: rows [yo0, yo1) of column band `band` advanced K steps (the
// fused kernel's register-path job with per-point coefficients).
template <int DT, int R, int PAT, int K, bool MASK>
__device__ __forceinline__ void vc2d_job(const VcParams<typename Traits<DT>::C> &p, int64_t band, int yo0, int yo1,
                                         int lane) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F2Geo<DT, R, K>;
    using Sh = Shape<2, R, PAT>;
    constexpr int V = G::V, W = G::W, H = G::H, BW = G::BW, NS = 2 * R;
    constexpr int U = lcm_c(NS, F2_PREF);
    constexpr uint32_t FULLM = (1u << V) - 1u;
    (void)W;
    const S *__restrict__ src = static_cast<const S *>(p.src);
    S *__restrict__ dst = static_cast<S *>(p.dst);
    const int nx = (int)p.g.n2, ny = (int)p.g.n1;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    const C bval = p.g.bval;
    const int xo0 = (int)band * BW;
    const int xl = xo0 - H + lane * V;
    const int yi0 = yo0 - R * K;
    const int nsp = round_up_c((yo1 - yo0) + 2 * R * K, U);
    uint32_t cmask = 0;
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (xl + v >= 0 && xl + v < nx) cmask |= 1u << v;
    const bool need_cmask = MASK && __any_sync(0xffffffffu, cmask != FULLM);
    bool keep[V];
#pragma unroll
    for (int v = 0; v < V; ++v) keep[v] = (cmask >> v) & 1u;
    const bool lane_out = (lane * V >= H) && (lane * V < H + BW);
    C pre[F2_PREF][V];
#pragma unroll
    for (int q = 0; q < F2_PREF; ++q)
        load_row_reg<DT, false>(src, nx, ny, !dir, bval, yi0 + q, xl, p.vec_ok != 0, pre[q]);
    C P[K][NS][V];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int m = 0; m < NS; ++m)
#pragma unroll
            for (int v = 0; v < V; ++v) P[s][m][v] = C(0);
    // the evaluation index of each (o_y, o_x) term, and the first term of a row
    constexpr int FOX = PAT == STENCIL_BOX ? -R : 0;
    for (int i0 = 0; i0 < nsp; i0 += U) {
#pragma unroll
        for (int ph = 0; ph < U; ++ph) {
            const int yin = yi0 + i0 + ph;
            C cur[V];
#pragma unroll
            for (int v = 0; v < V; ++v) cur[v] = pre[ph % F2_PREF][v];
            load_row_reg<DT, false>(src, nx, ny, !dir, bval, yin + F2_PREF, xl, p.vec_ok != 0, pre[ph % F2_PREF]);
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
                const int J = yin - s * R;   // the incoming level-s row
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
                // target row Y = J - oy takes the (o_y, o_x) terms with its own
                // coefficients c_(oy,ox)[Y]
#pragma unroll
                for (int oy = R; oy >= -R; --oy) {
                    const int m = R - oy;   // Y = J - R + m
#pragma unroll
                    for (int ox = -R; ox <= R; ++ox) {
                        if (!Sh::inc(0, oy, ox)) continue;
                        C cf[V];
                        vc_coef<DT>(p, p.ci[Sh::widx(0, oy, ox)], J - oy, xl, cf);
                        if (m == 0) vc_term<C, V, false>(cf, &ext[R + ox], emit);
                        else if (m < NS) vc_term<C, V, false>(cf, &ext[R + ox], P[s][(ph + m) % NS]);
                        else if (ox == FOX) vc_term<C, V, true>(cf, &ext[R + ox], P[s][s0]);
                        else vc_term<C, V, false>(cf, &ext[R + ox], P[s][s0]);
                    }
                }
                if constexpr (MASK) {
                    const int ye = J - R;
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
            const int yout = yin - K * R;
            if (yout >= yo0 && yout < yo1 && lane_out) {
                S *rowp = dst + (int64_t)yout * nx;
                if (p.vec_ok && xl + V <= nx) {
                    stvec<DT>(rowp + xl, cur);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (xl + v < nx) rowp[xl + v] = from_c<S>(cur[v]);
                }
            }
        }
    }
}

template <int DT, int R, int PAT, int K>
__global__ void __launch_bounds__(F2_NW * 32) vc2d_kernel(const __grid_constant__ VcParams<typename Traits<DT>::C> p) {
    using G = F2Geo<DT, R, K>;
    const int lane = threadIdx.x & 31;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    const int nx = (int)p.g.n2, ny = (int)p.g.n1;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&p.ctl->ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)p.jobs) break;
        const int64_t band = (int64_t)(t % p.bands), chunk = (int64_t)(t / p.bands);
        const int yo0 = (int)(chunk * p.Ly), yo1 = (int)std::min<int64_t>(yo0 + p.Ly, ny);
        const int xw0 = (int)band * G::BW - G::H;
        const bool interior = !dir || (xw0 >= 0 && xw0 + G::W <= nx && yo0 - R * K >= 0 && yo1 + R * K <= ny);
        if (interior) vc2d_job<DT, R, PAT, K, false>(p, band, yo0, yo1, lane);
        else vc2d_job<DT, R, PAT, K, true>(p, band, yo0, yo1, lane);
    }
    __syncwarp();
    if (lane == 0 && worker_exit_is_last(&p.ctl->exited, gridDim.x * F2_NW)) {
        p.ctl->ticket = 0ull;
        p.ctl->exited = 0u;
    }
}

constexpr int VC_KMAX = 4;   // fusion depths of the 2D variable-coefficient kernel (radius 1)
// radius 2 fuses up to 2 steps; radius 3 runs one step per launch
__host__ __device__ constexpr int vc_kmax(int r) { return r == 1 ? VC_KMAX : r == 2 ? 2 : 0; }

template <typename C> void vc_fill(const stencil_plan_s &P, VcParams<C> &p, const void *coef, const void *src,
                                   void *dst) {
    p.g.n0 = P.n[0];
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.src = src;
    p.dst = dst;
    p.coef = static_cast<const C *>(coef);
    p.N = P.npts;
    p.np = P.np;
    for (int j = 0; j < P.np; ++j) {
        p.ci[j] = (short)P.eval_to_compact[j];
        for (int a = 0; a < 3; ++a) p.off[j][a] = (signed char)P.off_eval[j][a];
    }
    const int v = (int)(16 / sizeof(C)) < 4 ? 2 : 4;
    p.vec_ok = (P.n[2] % v == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0) &&
               ((uintptr_t)coef % 16 == 0) && ((P.npts * sizeof(C)) % 16 == 0);
    p.ctl = static_cast<JobCtl *>(P.d_ctr);
    p.jobs = p.bands = p.Ly = 0;
}

template <int DT>
cudaError_t launch_vc_plain_t(const stencil_plan_s &P, const void *coef, const void *src, void *dst, cudaStream_t st) {
    VcParams<typename Traits<DT>::C> p;
    vc_fill(P, p, coef, src, dst);
    const int64_t items = P.n[0] * P.n[1] * ((P.n[2] + 3) / 4);
    int64_t blocks = (items + 255) / 256;
    if (blocks > (int64_t)P.sm_count * 16) blocks = (int64_t)P.sm_count * 16;
    vc_plain_kernel<DT><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(p);
    return cudaGetLastError();
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_vc2d_t(const stencil_plan_s &P, const void *coef, const void *src, void *dst, cudaStream_t st) {
    using G = F2Geo<DT, R, K>;
    VcParams<typename Traits<DT>::C> p;
    vc_fill(P, p, coef, src, dst);
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, vc2d_kernel<DT, R, PAT, K>, F2_NW * 32, 0);
    if (e != cudaSuccess) return e;
    const int64_t slots = (int64_t)P.sm_count * std::max(bps, 1) * F2_NW;
    const F2Tiling tl = f2_tiling(P.n[2], P.n[1], G::BW, R * K, slots, 2, P.tile_rows);
    p.bands = tl.bands;
    p.Ly = tl.Ly;
    p.jobs = tl.bands * tl.chunks;
    int64_t grid = (p.jobs + F2_NW - 1) / F2_NW;
    if (grid > (int64_t)P.sm_count * std::max(bps, 1)) grid = (int64_t)P.sm_count * std::max(bps, 1);
    vc2d_kernel<DT, R, PAT, K><<<(unsigned)grid, F2_NW * 32, 0, st>>>(p);
    return cudaGetLastError();
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_vc2d_kr(const stencil_plan_s &P, int k, const void *coef, const void *src, void *dst,
                           cudaStream_t st) {
    if constexpr (K > vc_kmax(R)) {
        return cudaErrorInvalidValue;
    } else {
        if (k == K) return launch_vc2d_t<DT, R, PAT, K>(P, coef, src, dst, st);
        return launch_vc2d_kr<DT, R, PAT, K + 1>(P, k, coef, src, dst, st);
    }
}

// one step (k = 0) or one fused 2D pass of k steps
template <int DT>
cudaError_t launch_vc_dt(const stencil_plan_s &P, int k, const void *coef, const void *src, void *dst,
                         cudaStream_t st) {
    if (k == 0) return launch_vc_plain_t<DT>(P, coef, src, dst, st);
    if (P.dim != 2) return cudaErrorInvalidValue;
    const bool box = P.pattern == STENCIL_BOX;
    switch (P.r) {
        case 1: return box ? launch_vc2d_kr<DT, 1, STENCIL_BOX, 1>(P, k, coef, src, dst, st)
                           : launch_vc2d_kr<DT, 1, STENCIL_STAR, 1>(P, k, coef, src, dst, st);
        case 2: return box ? launch_vc2d_kr<DT, 2, STENCIL_BOX, 1>(P, k, coef, src, dst, st)
                           : launch_vc2d_kr<DT, 2, STENCIL_STAR, 1>(P, k, coef, src, dst, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_vc_F32(const stencil_plan_s &, int, const void *, const void *, void *, cudaStream_t);
cudaError_t launch_vc_F64(const stencil_plan_s &, int, const void *, const void *, void *, cudaStream_t);
cudaError_t launch_vc_I32(const stencil_plan_s &, int, const void *, const void *, void *, cudaStream_t);

}  // namespace sg
