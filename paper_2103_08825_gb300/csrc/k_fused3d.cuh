// k_fused3d.cuh -- 3D Jacobi sweep with K time steps fused per pass,
// streaming along z (the outermost dimension).
//
// The paper's time-loop unroll-and-jam (Section 3.3, Algorithm 1) advances a
// vector set k levels while it streams past, keeping older levels in
// registers; its tiling (Section 3.4) extends the same scheme to 2D and 3D
// because only the unit-stride dimension is special.  Here a CTA owns an
// xy window of (W x WY) points and streams the planes of a z range:
//
//   threads   16 warps stacked in y, each warp RY = 2 rows of the window,
//             each lane V contiguous x values of those rows;
//   levels    every incoming plane of level s adds its terms to the 2r
//             partial planes of level s+1 it touches (registers); the plane
//             that receives its last term is emitted as level s+1's input;
//   in-plane  x-neighbours by warp shuffle; y-neighbours inside a warp are in
//             registers, the r rows beyond a warp's edges are exchanged with
//             the warps above and below through shared memory (one barrier
//             per level); level-0 planes are read straight from the stage;
//   input     PROD_TMA: warp 0 lane 0 loads whole window planes with 3D TMA
//             into an 8-stage ring (mbarrier completion, bounded waits);
//             PROD_CPASYNC: every thread copies its share of the plane with
//             cp.async, indices wrapped (periodic grids, unaligned rows);
//   halo      the window's outer H >= rK columns and rK rows are recomputed
//             (overlapped tiling); a z range reads rK planes each side;
//   order     one multiply then FMAs in lexicographic (o_z, o_y, o_x) order,
//             identical to the plain kernel: every K is bit-identical.
#pragma once

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

constexpr int F3_NWY = 16;               // warps per CTA, stacked in y
constexpr int F3_RY = 2;                 // window rows per warp
constexpr int F3_WY = F3_NWY * F3_RY;    // window rows
constexpr int F3_STAGES = 8;             // plane ring depth: ~112 KiB in flight per SM
constexpr int F3_THREADS = F3_NWY * 32;
enum { PROD3_TMA = 0, PROD3_CPASYNC = 1 };

template <int DT, int R, int K> struct F3Geo {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    static constexpr int V = Traits<DT>::V;
    static constexpr int W = 32 * V;
    static constexpr int AL = max_c(align_elems<DT>(), V);
    static constexpr int H = round_up_c(R * K, AL);
    static constexpr int BW = W - 2 * H;
    static constexpr int HY = R * K;
    static constexpr int BY = F3_WY - 2 * HY;
    static constexpr int PLANE = W * F3_WY;
    static constexpr int STAGE_BYTES = PLANE * (int)sizeof(S);
    static constexpr int XROWS = 2 * R;                              // edge rows a warp publishes
    static constexpr int XBUF_BYTES = 2 * F3_NWY * XROWS * W * (int)sizeof(C);
    static constexpr int SMEM = F3_STAGES * STAGE_BYTES + XBUF_BYTES + F3_STAGES * 8;
    static_assert(BW >= V && BY >= 1, "fusion depth too large for the window");
    static_assert(R <= V && R <= F3_RY, "halo must come from the neighbouring lane / warp");
};

template <typename C> struct F3Params {
    GridGeom<C> g;          // n0 = nz, n1 = ny, n2 = nx
    const void *src;
    void *dst;
    int64_t jobs, tiles_x, tiles_y, Lz;
    int vec_ok;
    int *status;
    JobCtl *ctl;            // job tickets (left at zero by the launch's last CTA)
    C w[125];               // evaluation order; up to the r = 2 box
};

template <typename C> struct F3MpParams {
    GridGeom<C> g;          // n0 = nz, n1 = ny, n2 = nx
    const void *src0;       // input of pass 0
    void *dst_even;         // output of the passes p with (passes - 1 - p) even (includes the last)
    void *dst_odd;
    int passes;
    int tiles_x, tiles_y, chunks, Lz;
    int vec_ok;
    int *status;
    MpCtl *ctl;             // ticket, abort flag, exit count
    int *done;              // [tiles]: passes each tile has finished
    int tiles;              // (all left at zero by the launch's last CTA)
    C w[125];
};

// V arithmetic values (16 or 32 bytes) to / from shared memory, 16-byte accesses
template <typename C, int V> __device__ __forceinline__ void st_shared_vec(C *p, const C *v) {
    static_assert((V * sizeof(C)) % 16 == 0, "16-byte units");
#pragma unroll
    for (int i = 0; i < (int)(V * sizeof(C)) / 16; ++i)
        reinterpret_cast<uint4 *>(p)[i] = reinterpret_cast<const uint4 *>(v)[i];
}
template <typename C, int V> __device__ __forceinline__ void ld_shared_vec(const C *p, C *v) {
#pragma unroll
    for (int i = 0; i < (int)(V * sizeof(C)) / 16; ++i)
        reinterpret_cast<uint4 *>(v)[i] = reinterpret_cast<const uint4 *>(p)[i];
}

__device__ __forceinline__ void cp_async4(void *smem, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copy window plane z (virtual, wrapped or boundary) into a stage, every
// thread a share, with cp.async (4-byte elements) or plain stores of the
// boundary value.  Used for periodic grids and rows TMA cannot address.  A
// thread copies the same 16-byte column chunk of several rows; a chunk that
// lies outside a periodic grid is wrapped by one extent, and when the grid's
// rows are 16-byte multiples it is still one aligned 16-byte copy.
template <int DT>
__device__ __forceinline__ void plane_copy_async(typename Traits<DT>::S *stage, const typename Traits<DT>::S *src,
                                                 int64_t nx, int64_t ny, int64_t nz, bool periodic,
                                                 typename Traits<DT>::C bval, int64_t xw0, int64_t yw0, int64_t z,
                                                 bool vec_ok) {
    using S = typename Traits<DT>::S;
    using G = F3Geo<DT, 1, 1>;
    constexpr int W = G::W;
    constexpr int VE = 16 / (int)sizeof(S);   // elements per 16-byte copy
    constexpr int TPR = W / VE;               // threads per window row
    constexpr int RSTEP = F3_THREADS / TPR;   // rows per sweep of the block
    static_assert(W % VE == 0 && F3_THREADS % TPR == 0, "chunking");
    bool zin = z >= 0 && z < nz;
    if (!zin && periodic) { z = wrap_idx(z, nz); zin = true; }
    const int col = (int)(threadIdx.x % TPR) * VE;
    const int64_t x0 = xw0 + col;
    int64_t xs = x0;
    bool xin = x0 >= 0 && x0 + VE <= nx;
    if (!xin && periodic) {
        xs = x0 < 0 ? x0 + nx : x0 - nx;
        xin = xs >= 0 && xs + VE <= nx;
    }
    const bool fast = vec_ok && xin;
    for (int row = (int)(threadIdx.x / TPR); row < F3_WY; row += RSTEP) {
        int64_t y = yw0 + row;
        bool yin = y >= 0 && y < ny;
        if (!yin && periodic) {
            y = y < 0 ? y + ny : y - ny;
            if (y < 0 || y >= ny) y = wrap_idx(y, ny);
            yin = true;
        }
        S *d = stage + row * W + col;
        if (!(zin && yin)) {
#pragma unroll
            for (int q = 0; q < VE; ++q) d[q] = from_c<S>(bval);
            continue;
        }
        const S *rowp = src + (z * ny + y) * nx;
        if (fast) {
            cp_async16(d, rowp + xs);
        } else {
#pragma unroll
            for (int q = 0; q < VE; ++q) {
                int64_t x = x0 + q;
                if (x >= 0 && x < nx) {
                    if constexpr (sizeof(S) >= 4) cp_async4(d + q, rowp + x);
                    else d[q] = rowp[x];
                } else if (periodic) {
                    if constexpr (sizeof(S) >= 4) cp_async4(d + q, rowp + wrap_idx(x, nx));
                    else d[q] = rowp[wrap_idx(x, nx)];
                } else {
                    d[q] = from_c<S>(bval);
                }
            }
        }
    }
}

// One job: the output tile [xo0, xo0+BW) x [yo0, yo0+BY) for planes
// [zo0, zo1).  MASK: the window touches a Dirichlet boundary, so out-of-domain
// cells are reset at every level.  Returns false if a bounded wait gave up.
template <int DT, int R, int PAT, int K, int PROD, bool MASK>
__device__ __forceinline__ bool fused3d_job(const CUtensorMap *tmap, const typename Traits<DT>::S *__restrict__ src,
                                            typename Traits<DT>::S *__restrict__ dst, int64_t nx, int64_t ny,
                                            int64_t nz, bool dir, typename Traits<DT>::C bval,
                                            const typename Traits<DT>::C *wr, int64_t xo0, int64_t yo0,
                                            int64_t zo0, int64_t zo1, bool vec_ok, typename Traits<DT>::S *stages,
                                            typename Traits<DT>::C *xbuf, uint64_t *bars, uint32_t &gst, int &xpar,
                                            int lane, int warp) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K>;
    using Sh = Shape<3, R, PAT>;
    constexpr int V = G::V, W = G::W, H = G::H, BW = G::BW, HY = G::HY, BY = G::BY;
    constexpr int RY = F3_RY, NS = 2 * R, NR = RY + 2 * R;   // NR: rows incl. y-halo
    constexpr int U = NS;                                    // z unroll: partial-plane slots repeat every 2R
    constexpr uint32_t FULLM = (1u << V) - 1u;
    const int64_t xw0 = xo0 - H, xl = xw0 + (int64_t)lane * V;
    const int64_t yw0 = yo0 - HY;
    const int64_t zi0 = zo0 - (int64_t)R * K;
    const int nsteps = (int)(zo1 - zo0) + 2 * R * K;
    const int nsp = round_up_c(nsteps, U);
    // column mask of this lane, row masks of this warp's rows (incl. halo)
    uint32_t cmask = 0;
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (xl + v >= 0 && xl + v < nx) cmask |= 1u << v;
    const int row0 = warp * RY;                  // first own window row
    // columns outside the domain: only warps that hold some need the selects
    bool keep[V];
#pragma unroll
    for (int v = 0; v < V; ++v) keep[v] = (cmask >> v) & 1u;
    const bool need_cmask = MASK && __any_sync(0xffffffffu, cmask != FULLM);
    const bool lane_out = (lane * V >= H) && (lane * V < H + BW);

    // ---- prologue: first stages
    if constexpr (PROD == PROD3_TMA) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            for (int q = 0; q < F3_STAGES && q < nsp; ++q) {
                const uint32_t slot = (gst + q) % F3_STAGES;
                mbar_arrive_expect_tx(&bars[slot], G::STAGE_BYTES);
                tma_load_3d(stages + (size_t)slot * G::PLANE, tmap, &bars[slot], (int)xw0, (int)yw0,
                            (int)(zi0 + q));
            }
        }
    } else {
        for (int q = 0; q < F3_STAGES - 1; ++q) {
            if (q < nsp)
                plane_copy_async<DT>(stages + (size_t)((gst + q) % F3_STAGES) * G::PLANE, src, nx, ny, nz, !dir,
                                     bval, xw0, yw0, zi0 + q, vec_ok);
            cp_async_commit();
        }
    }

    C P[K][NS][RY][V];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int m = 0; m < NS; ++m)
#pragma unroll
            for (int j = 0; j < RY; ++j)
#pragma unroll
                for (int v = 0; v < V; ++v) P[s][m][j][v] = C(0);

    bool bad = false;
    int ibad = 0;   // the plane whose stage a bounded wait gave up on
    for (int i0 = 0; i0 < nsp; i0 += U) {
#pragma unroll
        for (int ph = 0; ph < U; ++ph) {
            const int i = i0 + ph;
            const int64_t zin = zi0 + i;
            const uint32_t slot = (gst + i) % F3_STAGES;
            // ---- A: stage of plane zin ready
            if constexpr (PROD == PROD3_TMA) {
                const bool ok = mbar_wait_bounded(&bars[slot], ((gst + i) / F3_STAGES) & 1u);
                if (__syncthreads_or(!ok)) { bad = true; ibad = i; break; }
            } else {
                cp_async_wait<F3_STAGES - 2>();
                __syncthreads();
                if (i + F3_STAGES - 1 < nsp)
                    plane_copy_async<DT>(stages + (size_t)((gst + i + F3_STAGES - 1) % F3_STAGES) * G::PLANE, src,
                                         nx, ny, nz, !dir, bval, xw0, yw0, zin + F3_STAGES - 1, vec_ok);
                cp_async_commit();
            }
            // ---- B: level-0 rows row0-R .. row0+RY-1+R of this plane
            C inc[NR][V];
            {
                const S *pl = stages + (size_t)slot * G::PLANE;
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    int wrow = row0 - R + j;
                    wrow = wrow < 0 ? 0 : (wrow >= F3_WY ? F3_WY - 1 : wrow);   // beyond the window: halo garbage
                    ldsvec<DT>(pl + wrow * W + lane * V, inc[j]);
                }
                if constexpr (MASK) {
                    if ((uint32_t)zin >= (uint32_t)nz) {              // plane outside: uniform
#pragma unroll
                        for (int j = 0; j < NR; ++j)
#pragma unroll
                            for (int v = 0; v < V; ++v) inc[j][v] = bval;
                    } else {
#pragma unroll
                        for (int j = 0; j < NR; ++j) {
                            const int y = (int)yw0 + row0 - R + j;    // warp-uniform
                            if ((uint32_t)y >= (uint32_t)ny) {
#pragma unroll
                                for (int v = 0; v < V; ++v) inc[j][v] = bval;
                            } else if (need_cmask) {
#pragma unroll
                                for (int v = 0; v < V; ++v) inc[j][v] = keep[v] ? inc[j][v] : bval;
                            }
                        }
                    }
                }
            }
            if constexpr (K == 1) {
                __syncthreads();   // every warp has read the stage: refill it now
                if constexpr (PROD == PROD3_TMA) {
                    if (threadIdx.x == 0 && i + F3_STAGES < nsp) {
                        fence_proxy_async_smem();
                        const uint32_t g = gst + i + F3_STAGES, sl2 = g % F3_STAGES;
                        mbar_arrive_expect_tx(&bars[sl2], G::STAGE_BYTES);
                        tma_load_3d(stages + (size_t)sl2 * G::PLANE, tmap, &bars[sl2], (int)xw0, (int)yw0,
                                    (int)(zi0 + i + F3_STAGES));
                    }
                }
            }
            // ---- C: K levels
#pragma unroll
            for (int s = 0; s < K; ++s) {
                C emit[RY][V];
                // x-extended rows (star: only the own rows need x-neighbours)
                C ext[NR][V + 2 * R];
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    const bool need = (PAT == STENCIL_BOX) || (j >= R && j < R + RY);
#pragma unroll
                    for (int v = 0; v < V; ++v) ext[j][R + v] = inc[j][v];
                    if (need) {
#pragma unroll
                        for (int qq = 0; qq < R; ++qq) {
                            ext[j][R - 1 - qq] = __shfl_up_sync(0xffffffffu, inc[j][V - 1 - qq], 1);
                            ext[j][R + V + qq] = __shfl_down_sync(0xffffffffu, inc[j][qq], 1);
                        }
                    }
                }
                const int s0 = ph % NS;
                // complete plane J - R: o_z = +R terms
#pragma unroll
                for (int j = 0; j < RY; ++j)
#pragma unroll
                    for (int v = 0; v < V; ++v) emit[j][v] = P[s][s0][j][v];
#pragma unroll
                for (int oy = -R; oy <= R; ++oy)
#pragma unroll
                    for (int ox = -R; ox <= R; ++ox) {
                        if (!Sh::inc(R, oy, ox)) continue;
                        const C w = wr[Sh::widx(R, oy, ox)];
#pragma unroll
                        for (int j = 0; j < RY; ++j) row_fma_s<C, V>(w, &ext[j + R + oy][R + ox], emit[j]);
                    }
                // planes J - R + m take their o_z = R - m terms
#pragma unroll
                for (int m = 1; m < NS; ++m) {
                    const int oz = R - m, sl = (ph + m) % NS;
#pragma unroll
                    for (int oy = -R; oy <= R; ++oy)
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox) {
                            if (!Sh::inc(oz, oy, ox)) continue;
                            const C w = wr[Sh::widx(oz, oy, ox)];
#pragma unroll
                            for (int j = 0; j < RY; ++j) row_fma_s<C, V>(w, &ext[j + R + oy][R + ox], P[s][sl][j]);
                        }
                }
                // start plane J + R: o_z = -R terms, first one a multiply
                {
                    bool first = true;
#pragma unroll
                    for (int oy = -R; oy <= R; ++oy)
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox) {
                            if (!Sh::inc(-R, oy, ox)) continue;
                            const C w = wr[Sh::widx(-R, oy, ox)];
#pragma unroll
                            for (int j = 0; j < RY; ++j) {
                                if (first) row_mul_s<C, V>(w, &ext[j + R + oy][R + ox], P[s][s0][j]);
                                else row_fma_s<C, V>(w, &ext[j + R + oy][R + ox], P[s][s0][j]);
                            }
                            first = false;
                        }
                }
                // emitted plane index: Dirichlet cells keep the boundary value
                const int ze = (int)zin - (s + 1) * R;
                if constexpr (MASK) {
                    if ((uint32_t)ze >= (uint32_t)nz) {                // plane outside: uniform
#pragma unroll
                        for (int j = 0; j < RY; ++j)
#pragma unroll
                            for (int v = 0; v < V; ++v) emit[j][v] = bval;
                    } else {
#pragma unroll
                        for (int j = 0; j < RY; ++j) {
                            const int y = (int)yw0 + row0 + j;         // warp-uniform
                            if ((uint32_t)y >= (uint32_t)ny) {
#pragma unroll
                                for (int v = 0; v < V; ++v) emit[j][v] = bval;
                            } else if (need_cmask) {
#pragma unroll
                                for (int v = 0; v < V; ++v) emit[j][v] = keep[v] ? emit[j][v] : bval;
                            }
                        }
                    }
                }
                if (s + 1 < K) {
                    // exchange the r edge rows with the warps above and below
                    C *xb = xbuf + (size_t)xpar * F3_NWY * G::XROWS * W;
#pragma unroll
                    for (int qq = 0; qq < R; ++qq) {
                        st_shared_vec<C, V>(xb + ((size_t)warp * G::XROWS + qq) * W + lane * V, emit[qq]);
                        st_shared_vec<C, V>(xb + ((size_t)warp * G::XROWS + R + qq) * W + lane * V, emit[RY - R + qq]);
                    }
                    __syncthreads();
                    if (s == 0 && PROD == PROD3_TMA && threadIdx.x == 0 && i + F3_STAGES < nsp) {
                        // every warp has read this plane's stage: refill it
                        fence_proxy_async_smem();
                        const uint32_t g = gst + i + F3_STAGES, sl2 = g % F3_STAGES;
                        mbar_arrive_expect_tx(&bars[sl2], G::STAGE_BYTES);
                        tma_load_3d(stages + (size_t)sl2 * G::PLANE, tmap, &bars[sl2], (int)xw0, (int)yw0,
                                    (int)(zi0 + i + F3_STAGES));
                    }
                    const int wa = warp > 0 ? warp - 1 : warp;
                    const int wb = warp + 1 < F3_NWY ? warp + 1 : warp;
#pragma unroll
                    for (int qq = 0; qq < R; ++qq) {
                        ld_shared_vec<C, V>(xb + ((size_t)wa * G::XROWS + R + qq) * W + lane * V, inc[qq]);
                        ld_shared_vec<C, V>(xb + ((size_t)wb * G::XROWS + qq) * W + lane * V, inc[R + RY + qq]);
                    }
#pragma unroll
                    for (int j = 0; j < RY; ++j)
#pragma unroll
                        for (int v = 0; v < V; ++v) inc[R + j][v] = emit[j][v];
                    xpar ^= 1;
                } else {
                    // level K: store this warp's rows of the output tile
                    if (ze >= zo0 && ze < zo1 && lane_out) {
#pragma unroll
                        for (int j = 0; j < RY; ++j) {
                            const int wrow = row0 + j;
                            const int64_t y = yw0 + wrow;
                            if (wrow >= HY && wrow < HY + BY && y < ny) {
                                S *rowp = dst + (ze * ny + y) * nx;
                                if (vec_ok && xl + V <= nx) {
                                    stvec<DT>(rowp + xl, emit[j]);
                                } else {
#pragma unroll
                                    for (int v = 0; v < V; ++v)
                                        if (xl + v < nx) rowp[xl + v] = from_c<S>(emit[j][v]);
                                }
                            }
                        }
                    }
                }
            }

        }
        if (bad) break;
    }
    if (bad) {
        if (threadIdx.x == 0) {
            // wait (bounded, about ten seconds per stage) for this CTA's
            // copies still in flight before its shared memory can be left
            // (the planes ibad .. ibad + F3_STAGES - 1 of the job were issued)
            for (int q = ibad; q < ibad + F3_STAGES && q < nsp; ++q) {
                const uint32_t g = gst + q;
                if (!mbar_drain(&bars[g % F3_STAGES], (g / F3_STAGES) & 1u)) break;
            }
        }
        __syncthreads();
        return false;
    }
    if constexpr (PROD == PROD3_CPASYNC) cp_async_wait<0>();
    __syncthreads();
    gst += (uint32_t)nsp;
    return true;
}

template <int DT, int R, int PAT, int K, int PROD>
__global__ void __launch_bounds__(F3_THREADS, 1)
    fused3d_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ F3Params<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K>;
    using Sh = Shape<3, R, PAT>;
    extern __shared__ __align__(128) unsigned char smem[];
    S *stages = reinterpret_cast<S *>(smem);
    C *xbuf = reinterpret_cast<C *>(smem + F3_STAGES * G::STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + F3_STAGES * G::STAGE_BYTES + G::XBUF_BYTES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nx = p.g.n2, ny = p.g.n1, nz = p.g.n0;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    if constexpr (PROD == PROD3_TMA) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < F3_STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
            prefetch_tmap(&tmap);
        }
    }
    __syncthreads();
    C wr[Sh::npts];
#pragma unroll
    for (int j = 0; j < Sh::npts; ++j) wr[j] = p.w[j];
    uint32_t gst = 0;   // planes consumed so far by this CTA (stage ring position)
    int xpar = 0;       // exchange-buffer parity
    __shared__ unsigned long long s_ticket;
    // jobs are taken dynamically (faster SMs take more); the first and last z
    // ranges (Dirichlet edges) come first
    const int64_t nch = p.jobs / (p.tiles_x * p.tiles_y);
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&p.ctl->ticket, 1ull);
        __syncthreads();
        const unsigned long long t = s_ticket;
        __syncthreads();
        if (t >= (unsigned long long)p.jobs) break;
        const int64_t job = (int64_t)t;
        const int64_t tx = job % p.tiles_x, rest = job / p.tiles_x;
        const int64_t ty = rest % p.tiles_y, tc = rest / p.tiles_y;
        const int64_t cz = nch < 2 ? tc : (tc == 0 ? 0 : tc == 1 ? nch - 1 : tc - 1);
        const int64_t xo0 = tx * G::BW, yo0 = ty * G::BY;
        const int64_t zo0 = cz * p.Lz, zo1 = zo0 + p.Lz < nz ? zo0 + p.Lz : nz;
        // windows inside the domain never meet a Dirichlet cell: no masking code
        const bool interior = !dir || (xo0 - G::H >= 0 && xo0 - G::H + G::W <= nx && yo0 - G::HY >= 0 &&
                                       yo0 - G::HY + F3_WY <= ny && zo0 - R * K >= 0 && zo1 + R * K <= nz);
        const bool ok = interior
            ? fused3d_job<DT, R, PAT, K, PROD, false>(&tmap, static_cast<const S *>(p.src), static_cast<S *>(p.dst), nx,
                                                     ny, nz, dir, p.g.bval, wr, xo0, yo0, zo0, zo1, p.vec_ok != 0,
                                                     stages, xbuf, bars, gst, xpar, lane, warp)
            : fused3d_job<DT, R, PAT, K, PROD, true>(&tmap, static_cast<const S *>(p.src), static_cast<S *>(p.dst), nx,
                                                    ny, nz, dir, p.g.bval, wr, xo0, yo0, zo0, zo1, p.vec_ok != 0,
                                                    stages, xbuf, bars, gst, xpar, lane, warp);
        if (!ok) {
            if (threadIdx.x == 0) record_status(p.status, kStatusTimeout);
            break;
        }
    }
    // (the job loop's exits are uniform across the CTA)
    if (threadIdx.x == 0 && worker_exit_is_last(&p.ctl->exited, gridDim.x)) {
        p.ctl->ticket = 0ull;
        p.ctl->exited = 0u;
    }
}

// All `passes` passes of K steps in one persistent launch (3D form of
// fused2d_mp_kernel): CTAs take (pass, tile) items from one ticket,
// pass-major and z-major within a pass; an item of pass p first waits until
// every tile whose output meets its input window (up to 3 x 3 x 3 tiles, one
// thread each) has finished pass p - 1; completion is published with release
// semantics after the CTA's stores.  Waits are bounded (about one second); a
// wait that gives up raises the abort flag and records STENCIL_ERR_TIMEOUT.
template <int DT, int R, int PAT, int K, int PROD>
__global__ void __launch_bounds__(F3_THREADS, 1)
    fused3d_mp_kernel(const __grid_constant__ CUtensorMap tm_src0, const __grid_constant__ CUtensorMap tm_even,
                      const __grid_constant__ CUtensorMap tm_odd,
                      const __grid_constant__ F3MpParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K>;
    using Sh = Shape<3, R, PAT>;
    extern __shared__ __align__(128) unsigned char smem[];
    S *stages = reinterpret_cast<S *>(smem);
    C *xbuf = reinterpret_cast<C *>(smem + F3_STAGES * G::STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + F3_STAGES * G::STAGE_BYTES + G::XBUF_BYTES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = (int)p.g.n2, ny = (int)p.g.n1, nz = (int)p.g.n0;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    if constexpr (PROD == PROD3_TMA) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < F3_STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
            prefetch_tmap(&tm_src0);
            prefetch_tmap(&tm_even);
            prefetch_tmap(&tm_odd);
        }
    }
    __syncthreads();
    MpCtl *ctl = p.ctl;
    int *done = p.done;
    C wr[Sh::npts];
#pragma unroll
    for (int j = 0; j < Sh::npts; ++j) wr[j] = p.w[j];
    uint32_t gst = 0;
    int xpar = 0;
    const int txy = p.tiles_x * p.tiles_y;
    const int jobs = txy * p.chunks;
    const unsigned long long items = (unsigned long long)jobs * (unsigned)p.passes;
    __shared__ unsigned long long s_ticket;
    __shared__ int s_abort;
    // the next ticket and the abort flag are fetched one job ahead
    unsigned long long t_next = 0;
    int ab_next = 0;
    if (threadIdx.x == 0) t_next = atomicAdd(&ctl->ticket, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            s_ticket = t_next;
            s_abort = ab_next;
        }
        __syncthreads();
        const unsigned long long t = s_ticket;
        const int ab = s_abort;
        __syncthreads();
        if (t >= items || ab) break;
        if (threadIdx.x == 0) {
            t_next = atomicAdd(&ctl->ticket, 1ull);
            ab_next = ld_relaxed(&ctl->abort);
        }
        const int pass = (int)(t / (unsigned)jobs), j = (int)(t % (unsigned)jobs);
        const int cz = j / txy, rest = j - cz * txy;
        const int ty = rest / p.tiles_x, tx = rest - ty * p.tiles_x;
        const int xo0 = tx * G::BW, yo0 = ty * G::BY;
        const int zo0 = cz * p.Lz, zo1 = zo0 + p.Lz < nz ? zo0 + p.Lz : nz;
        if (pass > 0) {
            const int xe = xo0 + G::BW < nx ? xo0 + G::BW : nx;
            const int ye = yo0 + G::BY < ny ? yo0 + G::BY : ny;
            const TileSpan sx = tile_span(xo0 - G::H, xe + G::H, nx, G::BW, !dir);
            const TileSpan sy = tile_span(yo0 - G::HY, ye + G::HY, ny, G::BY, !dir);
            const TileSpan sz = tile_span(zo0 - R * K, zo1 + R * K, nz, p.Lz, !dir);
            const int cx = sx.count(), cxy = cx * sy.count(), nd = cxy * sz.count();
            bool ok = true;
            for (int e = threadIdx.x; e < nd; e += F3_THREADS) {
                const int ex = sx.at(e % cx), ey = sy.at((e % cxy) / cx), ez = sz.at(e / cxy);
                ok = ok && wait_counter(&done[(ez * p.tiles_y + ey) * p.tiles_x + ex], pass, &ctl->abort);
            }
            // the barrier orders every thread's acquire before every thread's reads
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) {
                    atomicExch(&ctl->abort, 1);
                    record_status(p.status, kStatusTimeout);
                }
                break;
            }
            if constexpr (PROD == PROD3_TMA) {
                if (threadIdx.x == 0) fence_proxy_async_global();
            }
        }
        const bool from_even = ((p.passes - pass) & 1) == 0;   // pass - 1 wrote dst_even
        const S *src = static_cast<const S *>(pass == 0 ? p.src0 : from_even ? p.dst_even : p.dst_odd);
        const CUtensorMap *tm = pass == 0 ? &tm_src0 : from_even ? &tm_even : &tm_odd;
        S *dst = static_cast<S *>(((p.passes - 1 - pass) & 1) == 0 ? p.dst_even : p.dst_odd);
        const bool interior = !dir || (xo0 - G::H >= 0 && xo0 - G::H + G::W <= nx && yo0 - G::HY >= 0 &&
                                       yo0 - G::HY + F3_WY <= ny && zo0 - R * K >= 0 && zo1 + R * K <= nz);
        const bool ok = interior
            ? fused3d_job<DT, R, PAT, K, PROD, false>(tm, src, dst, nx, ny, nz, dir, p.g.bval, wr, xo0, yo0, zo0, zo1,
                                                     p.vec_ok != 0, stages, xbuf, bars, gst, xpar, lane, warp)
            : fused3d_job<DT, R, PAT, K, PROD, true>(tm, src, dst, nx, ny, nz, dir, p.g.bval, wr, xo0, yo0, zo0, zo1,
                                                    p.vec_ok != 0, stages, xbuf, bars, gst, xpar, lane, warp);
        if (!ok) {
            if (threadIdx.x == 0) {
                atomicExch(&ctl->abort, 1);
                record_status(p.status, kStatusTimeout);
            }
            break;
        }
        // fused3d_job ends with a barrier after the CTA's last stores: publish
        if (threadIdx.x == 0) {
            if constexpr (PROD == PROD3_TMA) fence_proxy_async_global();
            red_release_add(&done[j], 1);
        }
    }
    // the last CTA out leaves the counters at zero for the next launch (the
    // loop's exits are uniform across the CTA)
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = worker_exit_is_last(&ctl->exited, gridDim.x);
    __syncthreads();
    if (s_last) {
        for (int i = threadIdx.x; i < p.tiles; i += F3_THREADS) done[i] = 0;
        if (threadIdx.x == 0) {
            ctl->ticket = 0ull;
            ctl->abort = 0;
            ctl->exited = 0u;
        }
    }
}

// z ranges: `lz` planes if set, else about three jobs per resident CTA;
// each range at least max(4 rK, 8) planes long
inline int64_t f3_lz(int64_t nz, int64_t tiles, int64_t slots, int rk, int lz) {
    const int64_t min_lz = 4 * rk > 8 ? 4 * rk : 8;
    if (lz > 0) return lz > min_lz ? (lz < nz ? lz : nz) : (min_lz < nz ? min_lz : nz);
    int64_t best_c = (3 * slots + tiles - 1) / tiles;
    if (best_c < 1) best_c = 1;
    const int64_t max_c = nz / min_lz > 1 ? nz / min_lz : 1;
    if (best_c > max_c) best_c = max_c;
    return (nz + best_c - 1) / best_c;
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_f3_t(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K>;
    F3Params<C> p;
    p.g.n0 = P.n[0];
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.src = src;
    p.dst = dst;
    p.status = P.d_status;
    p.ctl = static_cast<JobCtl *>(P.d_ctr);
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    const int64_t nx = P.n[2], ny = P.n[1], nz = P.n[0];
    p.vec_ok = (nx % G::V == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
    bool tma = P.bkind == STENCIL_DIRICHLET && ((nx * (int64_t)sizeof(S)) % 16 == 0) && ((uintptr_t)src % 16 == 0) &&
               nx < (1ll << 31) && ny < (1ll << 31) && nz < (1ll << 31);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (tma) {
        const int64_t dims[3] = {nx, ny, nz};
        const uint32_t box[3] = {(uint32_t)G::W, (uint32_t)F3_WY, 1u};
        tma = make_tmap(&map, DT, 3, dims, box, src);
    }
    // cp.async path: 16-byte copies need 16-byte aligned rows
    if (!tma) p.vec_ok = p.vec_ok && ((nx * (int64_t)sizeof(S)) % 16 == 0);
    auto kern = tma ? fused3d_kernel<DT, R, PAT, K, PROD3_TMA> : fused3d_kernel<DT, R, PAT, K, PROD3_CPASYNC>;
    const int smem = G::SMEM;
    static bool attr_done[2] = {false, false};
    if (!attr_done[tma ? 0 : 1]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_done[tma ? 0 : 1] = true;
    }
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, F3_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    p.tiles_x = (nx + G::BW - 1) / G::BW;
    p.tiles_y = (ny + G::BY - 1) / G::BY;
    const int64_t tiles = p.tiles_x * p.tiles_y;
    const int64_t slots = (int64_t)P.sm_count * bps;
    // z ranges: about three jobs per resident CTA (taken dynamically)
    p.Lz = f3_lz(nz, tiles, slots, R * K, P.tile_rows);
    const int64_t chunks = (nz + p.Lz - 1) / p.Lz;
    p.jobs = tiles * chunks;
    int64_t grid = p.jobs < slots ? p.jobs : slots;
    kern<<<(unsigned)grid, F3_THREADS, smem, st>>>(map, p);
    return cudaGetLastError();
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_f3mp_t(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int passes,
                          cudaStream_t st) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K>;
    if (!fused3d_multi_ok(P, K) || passes < 1) return cudaErrorNotSupported;
    F3MpParams<C> p;
    p.g.n0 = P.n[0];
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.src0 = src0;
    p.dst_even = dst_even;
    p.dst_odd = dst_odd;
    p.passes = passes;
    p.status = P.d_status;
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    const int64_t nx = P.n[2], ny = P.n[1], nz = P.n[0];
    const bool al = ((uintptr_t)src0 % 16 == 0) && ((uintptr_t)dst_even % 16 == 0) && ((uintptr_t)dst_odd % 16 == 0);
    p.vec_ok = (nx % G::V == 0) && al;
    bool tma = P.bkind == STENCIL_DIRICHLET && ((nx * (int64_t)sizeof(S)) % 16 == 0) && al;
    CUtensorMap maps[3];
    memset(maps, 0, sizeof(maps));
    if (tma) {
        const int64_t dims[3] = {nx, ny, nz};
        const uint32_t box[3] = {(uint32_t)G::W, (uint32_t)F3_WY, 1u};
        const void *bases[3] = {src0, dst_even, dst_odd};
        for (int i = 0; i < 3 && tma; ++i) tma = make_tmap(&maps[i], DT, 3, dims, box, bases[i]);
    }
    if (!tma) p.vec_ok = p.vec_ok && ((nx * (int64_t)sizeof(S)) % 16 == 0);
    auto kern = tma ? fused3d_mp_kernel<DT, R, PAT, K, PROD3_TMA> : fused3d_mp_kernel<DT, R, PAT, K, PROD3_CPASYNC>;
    const int smem = G::SMEM;
    static bool attr_done[2] = {false, false};
    if (!attr_done[tma ? 0 : 1]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_done[tma ? 0 : 1] = true;
    }
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, F3_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    const int64_t tiles_x = (nx + G::BW - 1) / G::BW, tiles_y = (ny + G::BY - 1) / G::BY;
    const int64_t slots = (int64_t)P.sm_count * bps;
    const int64_t lz = f3_lz(nz, tiles_x * tiles_y, slots, R * K, P.tile_rows);
    const int64_t chunks = (nz + lz - 1) / lz;
    const int64_t tiles = tiles_x * tiles_y * chunks;
    if (tiles >= (1ll << 28)) return cudaErrorNotSupported;
    p.tiles_x = (int)tiles_x;
    p.tiles_y = (int)tiles_y;
    p.chunks = (int)chunks;
    p.Lz = (int)lz;
    p.tiles = (int)tiles;
    e = ensure_mp_state(P, tiles, st);
    if (e != cudaSuccess) return e;
    p.ctl = static_cast<MpCtl *>(P.d_mp);
    p.done = reinterpret_cast<int *>(static_cast<char *>(P.d_mp) + sizeof(MpCtl));
    const int64_t jobs = tiles * passes;
    const int64_t grid = jobs < slots ? jobs : slots;
    kern<<<(unsigned)grid, F3_THREADS, smem, st>>>(maps[0], maps[1], maps[2], p);
    return cudaGetLastError();
}

template <int DT> constexpr int f3_kmax(int r) { return r == 1 ? 4 : 2; }

template <int DT, int R, int PAT>
cudaError_t launch_f3mp_k(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                          cudaStream_t st) {
    switch (k) {
        case 1: return launch_f3mp_t<DT, R, PAT, 1>(P, src0, de, dof, passes, st);
        case 2: return launch_f3mp_t<DT, R, PAT, 2>(P, src0, de, dof, passes, st);
        case 3: if constexpr (R == 1) return launch_f3mp_t<DT, R, PAT, 3>(P, src0, de, dof, passes, st); break;
        case 4: if constexpr (R == 1) return launch_f3mp_t<DT, R, PAT, 4>(P, src0, de, dof, passes, st); break;
    }
    return cudaErrorInvalidValue;
}

template <int DT>
cudaError_t launch_f3mp_dt(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                           cudaStream_t st) {
    const bool box = P.pattern == STENCIL_BOX;
    if (P.r == 1) return box ? launch_f3mp_k<DT, 1, STENCIL_BOX>(P, src0, de, dof, k, passes, st)
                             : launch_f3mp_k<DT, 1, STENCIL_STAR>(P, src0, de, dof, k, passes, st);
    if (P.r == 2) return box ? launch_f3mp_k<DT, 2, STENCIL_BOX>(P, src0, de, dof, k, passes, st)
                             : launch_f3mp_k<DT, 2, STENCIL_STAR>(P, src0, de, dof, k, passes, st);
    return cudaErrorInvalidValue;
}

template <int DT, int R, int PAT>
cudaError_t launch_f3_k(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (k) {
        case 1: return launch_f3_t<DT, R, PAT, 1>(P, src, dst, st);
        case 2: return launch_f3_t<DT, R, PAT, 2>(P, src, dst, st);
        case 3: if constexpr (R == 1) return launch_f3_t<DT, R, PAT, 3>(P, src, dst, st); break;
        case 4: if constexpr (R == 1) return launch_f3_t<DT, R, PAT, 4>(P, src, dst, st); break;
    }
    return cudaErrorInvalidValue;
}

template <int DT>
cudaError_t launch_f3_dt(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    const bool box = P.pattern == STENCIL_BOX;
    if (P.r == 1) return box ? launch_f3_k<DT, 1, STENCIL_BOX>(P, src, dst, k, st)
                             : launch_f3_k<DT, 1, STENCIL_STAR>(P, src, dst, k, st);
    if (P.r == 2) return box ? launch_f3_k<DT, 2, STENCIL_BOX>(P, src, dst, k, st)
                             : launch_f3_k<DT, 2, STENCIL_STAR>(P, src, dst, k, st);
    return cudaErrorInvalidValue;
}

}  // namespace sg
