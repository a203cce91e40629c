// k_fused3d.cuh -- 3D Jacobi sweep with K time steps fused per pass,
// streaming along z (the outermost dimension).
//
// The paper's time-loop unroll-and-jam (Section 3.3, Algorithm 1) advances a
// vector set k levels while it streams past, keeping older levels in
// registers ("vrl"); its tiling (Section 3.4) extends the scheme to 2D and 3D.
// Here a CTA owns an xy window of W x WY points and streams the planes of a z
// range through it:
//
//   threads   each half-warp (16 lanes x V contiguous values = W columns)
//             owns RY consecutive rows of the 64-row window, so a warp holds
//             2 RY rows and the CTA 32 / RY warps (RY = 2 or 4);
//   levels    every incoming plane of level s adds its terms to the 2r
//             partial planes of level s+1 it touches (registers); the plane
//             that receives its last term is emitted as level s+1's input;
//   in-plane  x-neighbours by shuffles within the half-warp; y-neighbours
//             from shared memory: level-0 rows straight from the TMA stage,
//             level s+1 rows from an exchange plane every half-warp writes
//             its emitted rows into (one CTA barrier per level);
//   input     PROD3_TMA: one thread loads whole window planes with 3D TMA
//             into an 8-stage ring (mbarrier completion, bounded waits);
//             PROD3_CPASYNC: every thread copies its share of the plane with
//             cp.async, indices wrapped (periodic grids, unaligned rows);
//   tiling    overlapped (the window recomputes an r k halo), but on a
//             Dirichlet grid a window never extends past the domain: the
//             first tile of an axis starts at 0 and the last ends at n, so the
//             boundary side needs no recomputed halo -- its neighbours are the
//             boundary value.  Interior tiles carry H >= r k halo columns
//             (16-byte aligned for TMA) and r k halo rows each side;
//   order     one multiply then FMAs in lexicographic (o_z, o_y, o_x) order,
//             identical to the plain kernel: every K is bit-identical.
#pragma once

#include <string.h>

#include <type_traits>

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

constexpr int F3_WY = 64;                // window rows: 32 / RY warps of two RY-row half-warps
constexpr int F3_LX = 16;                // lanes along x: a half-warp spans the window's width
constexpr int F3_STAGES = 8;             // plane ring depth (a power of two: cheap ring indices)
enum { PROD3_TMA = 0, PROD3_CPASYNC = 1 };

template <int DT, int R, int K, int RY> struct F3Geo {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    static constexpr int V = Traits<DT>::V;
    static constexpr int W = F3_LX * V;                              // window columns
    static constexpr int WY = F3_WY;                                 // window rows
    static constexpr int NW = F3_WY / (2 * RY);                      // warps per CTA
    static constexpr int THREADS = NW * 32;
    static constexpr int AL = max_c(align_elems<DT>(), V);
    static constexpr int H = round_up_c(R * K, AL);                  // x halo of an interior tile
    static constexpr int HY = R * K;                                 // y halo
    // a stage slot or exchange plane holds the window's WY rows between R
    // guard rows above and R below that keep the boundary value
    static constexpr int WYG = WY + 2 * R;
    static constexpr int SLOT = W * WYG;                             // elements
    static constexpr int SLOT_BYTES = SLOT * (int)sizeof(S);
    static constexpr int TMA_BYTES = W * WY * (int)sizeof(S);        // one window plane
    static constexpr int XPLANE = SLOT;
    static constexpr int XBUF_BYTES = 2 * XPLANE * (int)sizeof(C);   // exchange plane, double-buffered
    static constexpr int SMEM = F3_STAGES * SLOT_BYTES + XBUF_BYTES + F3_STAGES * 8;
    static_assert((R * W * (int)sizeof(S)) % 128 == 0 && SLOT_BYTES % 128 == 0, "TMA destination alignment");
    static_assert(W - 2 * H >= V && WY - 2 * HY >= 1, "fusion depth too large for the window");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Tiling of one axis.  bnd (a Dirichlet axis longer than the window): tile 0
// outputs [0, F) from the window [0, W); tiles 1 .. T-2 output B = W - 2H
// values each from a window starting H before their output; tile T-1 outputs
// the rest, up to n, from the window [n - W, n).  Otherwise uniform tiles of
// B values with windows starting `lo` before their output (H when periodic,
// 0 for a Dirichlet axis no longer than the window, which is one tile).
struct F3Axis {
    int n, W, H, T, F, B, lo, bnd;
};

inline F3Axis f3_axis(int64_t n, int W, int H, bool dirichlet) {
    F3Axis a{(int)n, W, H, 1, 0, W - 2 * H, H, 0};
    if (dirichlet && n > W) {
        a.bnd = 1;
        a.F = W - H;
        a.T = n <= 2 * a.F ? 2 : 2 + (int)((n - 2 * a.F + a.B - 1) / a.B);
        a.lo = H;
    } else if (dirichlet) {
        a.T = 1;
        a.B = (int)n;
        a.lo = 0;
    } else {
        a.T = (int)((n + a.B - 1) / a.B);
    }
    return a;
}

// output range [os, oe) and window start ws of tile t
__host__ __device__ __forceinline__ void f3_tile(const F3Axis &a, int t, int &os, int &oe, int &ws) {
    if (a.bnd) {
        os = t == 0 ? 0 : a.F + (t - 1) * a.B;
        oe = t == a.T - 1 ? a.n : a.F + t * a.B;
        ws = t == 0 ? 0 : (t == a.T - 1 ? a.n - a.W : os - a.H);
    } else {
        os = t * a.B;
        oe = os + a.B < a.n ? os + a.B : a.n;
        ws = os - a.lo;
    }
}

// The tiles whose outputs meet the coordinate range [lo, hi) (wrapped on a
// periodic axis; requires -n <= lo and hi <= 2n).
__host__ __device__ __forceinline__ TileSpan f3_span(const F3Axis &a, int lo, int hi, bool periodic) {
    if (!a.bnd) return tile_span(lo, hi, a.n, a.B, periodic);
    TileSpan s{0, 0, 0, 0, 0, 0};
    const int c0 = lo > 0 ? lo : 0, c1 = hi < a.n ? hi : a.n;
    if (c0 >= c1) return s;
    const int t0 = c0 < a.F ? 0 : 1 + (c0 - a.F) / a.B;
    const int t1 = c1 - 1 < a.F ? 0 : 1 + (c1 - 1 - a.F) / a.B;
    s.a0 = t0 < a.T - 1 ? t0 : a.T - 1;
    s.n0 = (t1 < a.T - 1 ? t1 : a.T - 1) + 1 - s.a0;
    return s;
}

template <typename C> struct F3Params {
    GridGeom<C> g;          // n0 = nz, n1 = ny, n2 = nx
    const void *src;
    void *dst;
    F3Axis ax, ay;
    int chunks, Lz;
    long long jobs;
    int vec_ok;
    int *status;
    JobCtl *ctl;            // job tickets (left at zero by the launch's last CTA)
    void *lv[4];            // ALL: levels 1 .. K - 1 of the pass are stored here too
    C w[kMaxPts];           // evaluation order (read from the constant bank)
};

template <typename C> struct F3MpParams {
    GridGeom<C> g;          // n0 = nz, n1 = ny, n2 = nx
    const void *src0;       // input of pass 0
    void *dst_even;         // output of the passes p with (passes - 1 - p) even (includes the last)
    void *dst_odd;
    int passes;
    F3Axis ax, ay;
    int chunks, Lz;
    int vec_ok;
    int *status;
    MpCtl *ctl;             // ticket, abort flag, exit count
    int *done;              // [tiles]: passes each tile has finished
    int tiles;              // (all left at zero by the launch's last CTA)
    C w[kMaxPts];
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


// Copy window plane z (virtual, wrapped or boundary) into a stage, every
// thread a share, with 16-byte cp.async copies where a chunk is aligned and
// L2 loads element by element elsewhere, or stores of the boundary value.  Used for periodic grids and rows TMA cannot address.  A
// thread copies the same 16-byte column chunk of several rows; a chunk that
// lies outside a periodic grid is wrapped by one extent, and when the grid's
// rows are 16-byte multiples it is still one aligned 16-byte copy.
template <int DT, int W, int WY, int THREADS>
__device__ __forceinline__ void plane_copy_async(typename Traits<DT>::S *stage, const typename Traits<DT>::S *src,
                                                 int64_t nx, int64_t ny, int64_t nz, bool periodic,
                                                 typename Traits<DT>::C bval, int64_t xw0, int64_t yw0, int64_t z,
                                                 bool vec_ok) {
    using S = typename Traits<DT>::S;
    constexpr int VE = 16 / (int)sizeof(S);   // elements per 16-byte copy
    constexpr int TPR = W / VE;               // threads per window row
    constexpr int RSTEP = THREADS / TPR;      // rows per sweep of the block
    static_assert(W % VE == 0 && THREADS % TPR == 0, "chunking");
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
    for (int row = (int)(threadIdx.x / TPR); row < WY; row += RSTEP) {
        int64_t y = yw0 + row;
        bool yin = y >= 0 && y < ny;
        if (!yin && periodic) {
            y = wrap_idx(y, ny);
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
            // element by element through L2 (ld.global.cg): within a
            // persistent launch other SMs wrote these values, so no copy may
            // come from a stale L1 line
#pragma unroll
            for (int q = 0; q < VE; ++q) {
                const int64_t x = x0 + q;
                if (x >= 0 && x < nx) d[q] = __ldcg(rowp + x);
                else if (periodic) d[q] = __ldcg(rowp + wrap_idx(x, nx));
                else d[q] = from_c<S>(bval);
            }
        }
    }
}

// x-neighbours of a lane's V values: ext[R + v] = x[v], ext[R - 1 - q] the
// value q + 1 columns left of the lane's first column, ext[R + V + q] the
// value q + 1 columns right of its last, taken from the lane q / V + 1
// positions away within the half-warp.  Lanes at the half-warp's edge get
// their own value there (window-edge halo: garbage that never reaches a stored
// output, or -- MASK -- replaced by the boundary value when that column lies
// outside the domain).
template <typename C, int V, int R, bool MASK>
__device__ __forceinline__ void x_extend(const C *x, C *ext, const bool *lout, const bool *rout, C bval) {
#pragma unroll
    for (int v = 0; v < V; ++v) ext[R + v] = x[v];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int d = q / V + 1;
        C l = __shfl_up_sync(0xffffffffu, x[V - 1 - q % V], d, F3_LX);
        C r = __shfl_down_sync(0xffffffffu, x[q % V], d, F3_LX);
        if constexpr (MASK) {
            l = lout[q] ? bval : l;
            r = rout[q] ? bval : r;
        }
        ext[R - 1 - q] = l;
        ext[R + V + q] = r;
    }
}

// Boundary value into the guard rows of every stage slot and both exchange
// planes (rows that no copy and no exchange ever writes).  Once per launch,
// before the CTA's first job; the caller's barrier publishes it.
template <int DT, int R, int K, int RY>
__device__ __forceinline__ void f3_guard_init(typename Traits<DT>::S *stages, typename Traits<DT>::C *xbuf,
                                              typename Traits<DT>::C bval) {
    using G = F3Geo<DT, R, K, RY>;
    constexpr int W = G::W, GE = 2 * R * W;   // guard elements per slot
    for (int e = threadIdx.x; e < (F3_STAGES + 2) * GE; e += G::THREADS) {
        const int sl = e / GE, q = e - sl * GE;
        const int row = q / W < R ? q / W : q / W + G::WY, col = q % W;
        if (sl < F3_STAGES) stages[(size_t)sl * G::SLOT + row * W + col] = from_c<typename Traits<DT>::S>(bval);
        else xbuf[(size_t)(sl - F3_STAGES) * G::XPLANE + row * W + col] = bval;
    }
}

// One job: the output tile [osx, oex) x [osy, oey) x [zo0, zo1) from the
// window columns [wsx, wsx + W) and rows [wsy, wsy + WY), streaming the planes
// zo0 - rK .. zo1 + rK - 1.
//
// Boundary handling (MASK: the job reaches the Dirichlet boundary).  Windows
// never extend past the domain (boundary-aware tiling), so in the steady
// state the only values from outside are (a) rows just beyond the window --
// the slots' and exchange planes' guard rows, which hold the boundary value --
// and (b) columns just beyond the window, which the window-edge lanes take
// from the boundary value by a select after their shuffles.  Planes outside
// the domain occur only in the first and last 2rK planes of the stream (the
// TMA fills them with zeros, and the levels emit planes there); those
// iterations, and every iteration of a window larger than the grid
// (`small`), run a second instance of the loop body that resets every cell
// outside the domain to the boundary value at every level.  Returns false if
// a bounded wait gave up.
template <int DT, int R, int PAT, int K, int RY, int PROD, bool MASK, bool ALL = false>
__device__ __forceinline__ bool fused3d_job(const CUtensorMap *tmap, const typename Traits<DT>::S *__restrict__ src,
                                            typename Traits<DT>::S *__restrict__ dst, void *const *lv, int nx, int ny,
                                            int nz,
                                            bool dir, typename Traits<DT>::C bval, const typename Traits<DT>::C *wr,
                                            int wsx, int osx, int oex, int wsy, int osy, int oey, int zo0, int zo1,
                                            bool vec_ok, bool small, typename Traits<DT>::S *stages,
                                            typename Traits<DT>::C *xbuf, uint64_t *bars, uint32_t &gst, int lane,
                                            int warp) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K, RY>;
    using Sh = Shape<3, R, PAT>;
    constexpr int V = G::V, W = G::W, WY = G::WY, SLOT = G::SLOT;
    constexpr int NS = 2 * R, NR = RY + 2 * R;   // NR: rows a half-warp reads, with the y-halo
    constexpr int U = NS;                        // z unroll: partial-plane slots repeat every 2R
    constexpr int RK = R * K;
    // the first term of a plane (o_z = -R) in lexicographic order
    constexpr int FOY = PAT == STENCIL_BOX ? -R : 0, FOX = PAT == STENCIL_BOX ? -R : 0;
    const int l16 = lane & (F3_LX - 1);
    const int row0 = (warp * 2 + (lane >> 4)) * RY;   // first own window row
    const int xl = wsx + l16 * V;                     // first own column
    const int zi0 = zo0 - RK;
    const int nsteps = (zo1 - zo0) + 2 * RK;
    const int nsp = round_up_c(nsteps, U);
    // a thread's reads start at window row row0 - R = slot row row0
    const int rdoff = row0 * W + l16 * V;
    // neighbour columns outside the domain (window-edge lanes of an edge window)
    bool lout[R], rout[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        lout[q] = MASK && (xl - 1 - q < 0 || xl - 1 - q >= nx);
        rout[q] = MASK && (xl + V + q < 0 || xl + V + q >= nx);
    }
    // masked iterations: own columns and the NR rows read (bit j: window row
    // row0 - R + j) outside the domain
    bool keep[V];
#pragma unroll
    for (int v = 0; v < V; ++v) keep[v] = xl + v >= 0 && xl + v < nx;
    uint32_t yout_bits = 0;
#pragma unroll
    for (int j = 0; j < NR; ++j) yout_bits |= (unsigned)(wsy + row0 - R + j) >= (unsigned)ny ? 1u << j : 0u;
    // stores: rows of the output tile, whole vectors inside it
    uint32_t ystore = 0;
#pragma unroll
    for (int j = 0; j < RY; ++j) ystore |= (wsy + row0 + j >= osy && wsy + row0 + j < oey) ? 1u << j : 0u;
    const bool xvec = vec_ok && xl >= osx && xl + V <= oex;
    const bool xsome = !xvec && xl + V > osx && xl < oex;   // part of the lane's columns
    const int64_t orow = (int64_t)(wsy + row0) * nx + xl;   // own first row, plane 0
    const int64_t pstride = (int64_t)nx * ny;
    // this half-warp's rows of the output tile of plane ze into `base`
    auto store_rows = [&](S *base, int ze, const C (&rows)[RY][V]) {
        S *op = base + orow + (int64_t)ze * pstride;
#pragma unroll
        for (int j = 0; j < RY; ++j) {
            if (!((ystore >> j) & 1u)) continue;
            S *rp = op + (int64_t)j * nx;
            if (xvec) {
                stvec<DT>(rp, rows[j]);
            } else if (xsome) {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (xl + v >= osx && xl + v < oex) rp[v] = from_c<S>(rows[j][v]);
            }
        }
    };

    // ---- prologue: first stages
    if constexpr (PROD == PROD3_TMA) {
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            for (int q = 0; q < F3_STAGES && q < nsp; ++q) {
                const uint32_t slot = (gst + q) % F3_STAGES;
                mbar_arrive_expect_tx(&bars[slot], G::TMA_BYTES);
                tma_load_3d(stages + (size_t)slot * SLOT + R * W, tmap, &bars[slot], wsx, wsy, zi0 + q);
            }
        }
    } else {
        for (int q = 0; q < F3_STAGES - 1; ++q) {
            if (q < nsp)
                plane_copy_async<DT, W, WY, G::THREADS>(stages + (size_t)((gst + q) % F3_STAGES) * SLOT + R * W, src, nx, ny, nz,
                                            !dir, bval, wsx, wsy, zi0 + q, vec_ok);
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

    // A bounded wait that gives up is voted on at the level's first CTA
    // barrier; from then on the job only runs out its loop (no waits, copies
    // or stores) and returns false.
    bool bad = false;
    int ibad = 0;   // the plane whose stage a bounded wait gave up on

    // One unrolled group of U planes; ZM: the masked instance.
    auto group = [&](auto zm_tag, const int i0) {
        constexpr bool ZM = decltype(zm_tag)::value;
#pragma unroll
        for (int ph = 0; ph < U; ++ph) {
            const int i = i0 + ph;
            const int zin = zi0 + i;
            const uint32_t g = gst + (uint32_t)i, slot = g % F3_STAGES;
            // ---- A: stage of plane zin ready
            bool waitbad = false;
            if constexpr (PROD == PROD3_TMA) {
                if (!bad) waitbad = !mbar_wait_bounded(&bars[slot], (g / F3_STAGES) & 1u);
            } else {
                cp_async_wait<F3_STAGES - 2>();
                __syncthreads();
                if (i + F3_STAGES - 1 < nsp)
                    plane_copy_async<DT, W, WY, G::THREADS>(stages + (size_t)((g + F3_STAGES - 1) % F3_STAGES) * SLOT + R * W,
                                                src, nx, ny, nz, !dir, bval, wsx, wsy, zin + F3_STAGES - 1, vec_ok);
                cp_async_commit();
            }
            // ---- B: level-0 rows row0-R .. row0+RY-1+R of this plane
            C inc[NR][V];
            {
                const S *pl = stages + (size_t)slot * SLOT + rdoff;
#pragma unroll
                for (int j = 0; j < NR; ++j) ldsvec<DT>(pl + j * W, inc[j]);
                if constexpr (ZM) {
                    const bool zout = (unsigned)zin >= (unsigned)nz;
#pragma unroll
                    for (int j = 0; j < NR; ++j)
#pragma unroll
                        for (int v = 0; v < V; ++v)
                            inc[j][v] = (zout || ((yout_bits >> j) & 1u) || !keep[v]) ? bval : inc[j][v];
                }
            }
            if constexpr (K == 1) {
                // every warp has read the stage: refill it now
                if (__syncthreads_or(waitbad) && !bad) {
                    bad = true;
                    ibad = i;
                }
                if constexpr (PROD == PROD3_TMA) {
                    if (threadIdx.x == 0 && !bad && i + F3_STAGES < nsp) {
                        fence_proxy_async_smem();
                        const uint32_t g2 = g + F3_STAGES, sl2 = g2 % F3_STAGES;
                        mbar_arrive_expect_tx(&bars[sl2], G::TMA_BYTES);
                        tma_load_3d(stages + (size_t)sl2 * SLOT + R * W, tmap, &bars[sl2], wsx, wsy, zin + F3_STAGES);
                    }
                }
            }
            // ---- C: K levels.  inc: level-s rows of plane J = zin - sR.
#pragma unroll
            for (int s = 0; s < K; ++s) {
                const int s0 = ph % NS;   // slot of plane J - R (completed now), reused for J + R
                C emit[RY][V];
#pragma unroll
                for (int j = 0; j < RY; ++j)
#pragma unroll
                    for (int v = 0; v < V; ++v) emit[j][v] = P[s][s0][j][v];
                // source rows in ascending order, so that each target row gets
                // its terms in ascending (o_y, o_x) order within every o_z
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    const bool needx = PAT == STENCIL_BOX || (j >= R && j < R + RY);
                    C ext[V + 2 * R];
                    if (needx) {
                        x_extend<C, V, R, MASK>(inc[j], ext, lout, rout, bval);
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) ext[R + v] = inc[j][v];
                    }
#pragma unroll
                    for (int oy = -R; oy <= R; ++oy) {
                        const int jt = j - R - oy;   // target row
                        if (jt < 0 || jt >= RY) continue;
                        // o_z = +R: the last terms of plane J - R
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox)
                            if (Sh::inc(R, oy, ox)) row_fma_s<C, V>(wr[Sh::widx(R, oy, ox)], &ext[R + ox], emit[jt]);
                        // o_z = R - m: planes J - R + m (0 < m < 2R)
#pragma unroll
                        for (int m = 1; m < NS; ++m) {
                            const int oz = R - m, sl = (ph + m) % NS;
#pragma unroll
                            for (int ox = -R; ox <= R; ++ox)
                                if (Sh::inc(oz, oy, ox))
                                    row_fma_s<C, V>(wr[Sh::widx(oz, oy, ox)], &ext[R + ox], P[s][sl][jt]);
                        }
                        // o_z = -R: the first terms of plane J + R (first one a multiply)
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox) {
                            if (!Sh::inc(-R, oy, ox)) continue;
                            if (oy == FOY && ox == FOX) row_mul_s<C, V>(wr[Sh::widx(-R, oy, ox)], &ext[R + ox], P[s][s0][jt]);
                            else row_fma_s<C, V>(wr[Sh::widx(-R, oy, ox)], &ext[R + ox], P[s][s0][jt]);
                        }
                    }
                }
                // emitted plane ze = J - R; masked iterations: cells outside
                // the domain keep the boundary value
                const int ze = zin - (s + 1) * R;
                if constexpr (ZM) {
                    const bool zout = (unsigned)ze >= (unsigned)nz;
#pragma unroll
                    for (int j = 0; j < RY; ++j)
#pragma unroll
                        for (int v = 0; v < V; ++v)
                            emit[j][v] = (zout || ((yout_bits >> (R + j)) & 1u) || !keep[v]) ? bval : emit[j][v];
                }
                if (s + 1 < K) {
                    // publish the rows within R of the half-warp's edges (the
                    // only ones other half-warps read); read the R rows above
                    // and below -- another half-warp's or a guard row.  The
                    // parity alternates per exchange and, U (K - 1) being
                    // even, starts every group at 0.
                    C *xb = xbuf + ((ph * (K - 1) + s) & 1) * G::XPLANE + rdoff;
#pragma unroll
                    for (int j = 0; j < RY; ++j)
                        if (j < R || j >= RY - R) st_shared_vec<C, V>(xb + (R + j) * W, emit[j]);
                    if (s == 0) {
                        if (__syncthreads_or(waitbad) && !bad) {
                            bad = true;
                            ibad = i;
                        }
                        if constexpr (PROD == PROD3_TMA) {
                            if (threadIdx.x == 0 && !bad && i + F3_STAGES < nsp) {
                                // every warp has read this plane's stage: refill it
                                fence_proxy_async_smem();
                                const uint32_t g2 = g + F3_STAGES, sl2 = g2 % F3_STAGES;
                                mbar_arrive_expect_tx(&bars[sl2], G::TMA_BYTES);
                                tma_load_3d(stages + (size_t)sl2 * SLOT + R * W, tmap, &bars[sl2], wsx, wsy,
                                            zin + F3_STAGES);
                            }
                        }
                    } else {
                        __syncthreads();
                    }
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        ld_shared_vec<C, V>(xb + j * W, inc[j]);
                        ld_shared_vec<C, V>(xb + (R + RY + j) * W, inc[R + RY + j]);
                    }
#pragma unroll
                    for (int j = 0; j < RY; ++j)
#pragma unroll
                        for (int v = 0; v < V; ++v) inc[R + j][v] = emit[j][v];
                    if constexpr (ALL) {
                        // level s + 1 of the output tile, kept as well
                        if (!bad && ze >= zo0 && ze < zo1) store_rows(static_cast<S *>(lv[s]), ze, emit);
                    }
                } else if (!bad && ze >= zo0 && ze < zo1) {
                    // level K: store this half-warp's rows of the output tile
                    store_rows(dst, ze, emit);
                }
            }
        }
    };

    static_assert((U * (K - 1)) % 2 == 0, "exchange parity must restart every group");
    for (int i0 = 0; i0 < nsp; i0 += U) {
        if constexpr (MASK) {
            const int zlo = zi0 + i0;
            if (small || zlo < RK || zlo + U - 1 >= nz) group(std::true_type{}, i0);
            else group(std::false_type{}, i0);
        } else {
            group(std::false_type{}, i0);
        }
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

// A job of a Dirichlet grid whose window and z range stay strictly inside the
// domain never meets a boundary cell or neighbour: it runs without masking.
template <int W, int WY, int RK>
__device__ __forceinline__ bool f3_interior(bool dir, int nx, int ny, int nz, int wsx, int wsy, int zo0, int zo1) {
    return !dir || (wsx > 0 && wsx + W < nx && wsy > 0 && wsy + WY < ny && zo0 - RK >= 0 && zo1 + RK <= nz);
}

template <int DT, int R, int PAT, int K, int RY, int PROD, bool ALL = false>
__global__ void __launch_bounds__((F3Geo<DT, R, K, RY>::THREADS), 1)
    fused3d_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ F3Params<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K, RY>;
    extern __shared__ __align__(128) unsigned char smem[];
    S *stages = reinterpret_cast<S *>(smem);
    C *xbuf = reinterpret_cast<C *>(smem + F3_STAGES * G::SLOT_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + F3_STAGES * G::SLOT_BYTES + G::XBUF_BYTES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = (int)p.g.n2, ny = (int)p.g.n1, nz = (int)p.g.n0;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    if constexpr (PROD == PROD3_TMA) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < F3_STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
            prefetch_tmap(&tmap);
        }
    }
    f3_guard_init<DT, R, K, RY>(stages, xbuf, p.g.bval);
    __syncthreads();
    const C *wr = p.w;   // parameter space: the FMAs read the weights as constant operands
    const bool small = p.ax.n < G::W || p.ay.n < G::WY;   // the window is larger than the grid
    uint32_t gst = 0;    // planes consumed so far by this CTA (stage ring position)
    __shared__ unsigned long long s_ticket;
    // jobs are taken dynamically (faster SMs take more); the first and last z
    // ranges (Dirichlet edges) come first
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&p.ctl->ticket, 1ull);
        __syncthreads();
        const unsigned long long t = s_ticket;
        __syncthreads();
        if (t >= (unsigned long long)p.jobs) break;
        const int job = (int)t;
        const int tx = job % p.ax.T, rest = job / p.ax.T;
        const int ty = rest % p.ay.T, tc = rest / p.ay.T;
        const int nch = p.chunks;
        const int cz = nch < 2 ? tc : (tc == 0 ? 0 : tc == 1 ? nch - 1 : tc - 1);
        int osx, oex, wsx, osy, oey, wsy;
        f3_tile(p.ax, tx, osx, oex, wsx);
        f3_tile(p.ay, ty, osy, oey, wsy);
        const int zo0 = cz * p.Lz, zo1 = zo0 + p.Lz < nz ? zo0 + p.Lz : nz;
        const bool ok = f3_interior<G::W, G::WY, R * K>(dir, nx, ny, nz, wsx, wsy, zo0, zo1)
            ? fused3d_job<DT, R, PAT, K, RY, PROD, false, ALL>(&tmap, static_cast<const S *>(p.src), static_cast<S *>(p.dst), p.lv,
                                                          nx, ny, nz, dir, p.g.bval, wr, wsx, osx, oex, wsy, osy, oey,
                                                          zo0, zo1, p.vec_ok != 0, small, stages, xbuf, bars, gst, lane,
                                                          warp)
            : fused3d_job<DT, R, PAT, K, RY, PROD, true, ALL>(&tmap, static_cast<const S *>(p.src), static_cast<S *>(p.dst), p.lv,
                                                         nx, ny, nz, dir, p.g.bval, wr, wsx, osx, oex, wsy, osy, oey,
                                                         zo0, zo1, p.vec_ok != 0, small, stages, xbuf, bars, gst, lane,
                                                         warp);
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
// every tile whose output meets the dependency cone of its own output (its
// output extended by rK on every axis, wrapped on periodic axes; up to
// 3 x 3 x 3 tiles, one thread each) has finished pass p - 1; completion is
// published with release semantics after the CTA's stores.  Waits are bounded
// (about one second); a wait that gives up raises the abort flag and records
// STENCIL_ERR_TIMEOUT.
template <int DT, int R, int PAT, int K, int RY, int PROD>
__global__ void __launch_bounds__((F3Geo<DT, R, K, RY>::THREADS), 1)
    fused3d_mp_kernel(const __grid_constant__ CUtensorMap tm_src0, const __grid_constant__ CUtensorMap tm_even,
                      const __grid_constant__ CUtensorMap tm_odd,
                      const __grid_constant__ F3MpParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F3Geo<DT, R, K, RY>;
    extern __shared__ __align__(128) unsigned char smem[];
    S *stages = reinterpret_cast<S *>(smem);
    C *xbuf = reinterpret_cast<C *>(smem + F3_STAGES * G::SLOT_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + F3_STAGES * G::SLOT_BYTES + G::XBUF_BYTES);
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
    f3_guard_init<DT, R, K, RY>(stages, xbuf, p.g.bval);
    __syncthreads();
    MpCtl *ctl = p.ctl;
    int *done = p.done;
    const C *wr = p.w;
    const bool small = p.ax.n < G::W || p.ay.n < G::WY;   // the window is larger than the grid
    uint32_t gst = 0;
    const int txy = p.ax.T * p.ay.T;
    const int jobs = txy * p.chunks;
    const unsigned long long items = (unsigned long long)jobs * (unsigned)p.passes;
    constexpr int RK = R * K;
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
        const int ty = rest / p.ax.T, tx = rest - ty * p.ax.T;
        int osx, oex, wsx, osy, oey, wsy;
        f3_tile(p.ax, tx, osx, oex, wsx);
        f3_tile(p.ay, ty, osy, oey, wsy);
        const int zo0 = cz * p.Lz, zo1 = zo0 + p.Lz < nz ? zo0 + p.Lz : nz;
        if (pass > 0) {
            const TileSpan sx = f3_span(p.ax, osx - RK, oex + RK, !dir);
            const TileSpan sy = f3_span(p.ay, osy - RK, oey + RK, !dir);
            const TileSpan sz = tile_span(zo0 - RK, zo1 + RK, nz, p.Lz, !dir);
            const int cx = sx.count(), cxy = cx * sy.count(), nd = cxy * sz.count();
            bool ok = true;
            for (int e = threadIdx.x; e < nd; e += G::THREADS) {
                const int ex = sx.at(e % cx), ey = sy.at((e % cxy) / cx), ez = sz.at(e / cxy);
                ok = ok && wait_counter(&done[(ez * p.ay.T + ey) * p.ax.T + ex], pass, &ctl->abort);
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
        const bool ok = f3_interior<G::W, G::WY, RK>(dir, nx, ny, nz, wsx, wsy, zo0, zo1)
            ? fused3d_job<DT, R, PAT, K, RY, PROD, false>(tm, src, dst, nullptr, nx, ny, nz, dir, p.g.bval, wr, wsx, osx, oex,
                                                          wsy, osy, oey, zo0, zo1, p.vec_ok != 0, small, stages, xbuf,
                                                          bars, gst, lane, warp)
            : fused3d_job<DT, R, PAT, K, RY, PROD, true>(tm, src, dst, nullptr, nx, ny, nz, dir, p.g.bval, wr, wsx, osx, oex,
                                                         wsy, osy, oey, zo0, zo1, p.vec_ok != 0, small, stages, xbuf,
                                                         bars, gst, lane, warp);
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
        for (int i = threadIdx.x; i < p.tiles; i += G::THREADS) done[i] = 0;
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

// Rows per half-warp: 4 (8 warps, up to 255 registers a thread) for the
// radius-1 star at K = 4, where fewer barriers and shared-memory accesses per
// row outweigh the lower warp count; else 2 (16 warps, 128 registers).
template <int DT, int R, int PAT, int K> constexpr int f3_ry() {
    return R == 1 && PAT == STENCIL_STAR && K == 4 &&
                   K * 2 * R * 4 * Traits<DT>::V * (int)(sizeof(typename Traits<DT>::C) / 4) <= 128
               ? 4
               : 2;
}

template <typename Prm>
void f3_fill_common(const stencil_plan_s &P, Prm &p, int W, int H, int WY, int HY) {
    using C = std::remove_reference_t<decltype(p.w[0])>;
    p.g.n0 = P.n[0];
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.status = P.d_status;
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    const bool dir = P.bkind == STENCIL_DIRICHLET;
    p.ax = f3_axis(P.n[2], W, H, dir);
    p.ay = f3_axis(P.n[1], WY, HY, dir);
}

// x halo of a TMA-fed Dirichlet grid: with boundary-aware tiling the windows
// start at 0, at multiples of the tile width B = W - 2h and at n - W, so only
// B (and n, which TMA already needs) must be 16-byte multiples -- the halo
// itself need not be (a 4-column halo instead of 8 for 2-byte types).  The
// periodic and cp.async paths keep G::H, a 16-byte multiple (their windows
// start h before each tile).
inline int f3_hx(int rk, int W, int al) {
    int h = rk;
    while ((W - 2 * h) % al != 0) ++h;
    return h;
}

// lv (ALL): levels 1 .. K - 1 of the pass are also stored, level l into lv[l - 1]
template <int DT, int R, int PAT, int K, bool ALL = false>
cudaError_t launch_f3_t(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st,
                        void *const *lv = nullptr) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    constexpr int RY = f3_ry<DT, R, PAT, K>();
    using G = F3Geo<DT, R, K, RY>;
    F3Params<C> p;
    f3_fill_common(P, p, G::W, G::H, G::WY, G::HY);
    p.src = src;
    p.dst = dst;
    p.ctl = static_cast<JobCtl *>(P.d_ctr);
    for (int l = 0; l < 4; ++l) p.lv[l] = ALL && l < K - 1 ? lv[l] : nullptr;
    const int64_t nx = P.n[2], ny = P.n[1], nz = P.n[0];
    p.vec_ok = (nx % G::V == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
    for (int l = 0; l < K - 1; ++l) p.vec_ok = p.vec_ok && (!ALL || (uintptr_t)p.lv[l] % 16 == 0);
    bool tma = P.bkind == STENCIL_DIRICHLET && ((nx * (int64_t)sizeof(S)) % 16 == 0) && ((uintptr_t)src % 16 == 0);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (tma) {
        const int64_t dims[3] = {nx, ny, nz};
        const uint32_t box[3] = {(uint32_t)G::W, (uint32_t)G::WY, 1u};
        tma = make_tmap(&map, DT, 3, dims, box, src);
    }
    if (tma) f3_fill_common(P, p, G::W, f3_hx(R * K, G::W, G::AL), G::WY, G::HY);
    // cp.async path: 16-byte copies need 16-byte aligned rows
    if (!tma) p.vec_ok = p.vec_ok && ((nx * (int64_t)sizeof(S)) % 16 == 0);
    auto kern = tma ? fused3d_kernel<DT, R, PAT, K, RY, PROD3_TMA, ALL>
                    : fused3d_kernel<DT, R, PAT, K, RY, PROD3_CPASYNC, ALL>;
    const int smem = G::SMEM;
    static bool attr_done[2] = {false, false};
    if (!attr_done[tma ? 0 : 1]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_done[tma ? 0 : 1] = true;
    }
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, G::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    const int64_t tiles = (int64_t)p.ax.T * p.ay.T;
    const int64_t slots = (int64_t)P.sm_count * bps;
    // z ranges: about three jobs per resident CTA (taken dynamically)
    p.Lz = (int)f3_lz(nz, tiles, slots, R * K, P.tile_rows);
    p.chunks = (int)((nz + p.Lz - 1) / p.Lz);
    p.jobs = tiles * p.chunks;
    const int64_t grid = p.jobs < slots ? p.jobs : slots;
    kern<<<(unsigned)grid, G::THREADS, smem, st>>>(map, p);
    return cudaGetLastError();
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_f3mp_t(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int passes,
                          cudaStream_t st) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    constexpr int RY = f3_ry<DT, R, PAT, K>();
    using G = F3Geo<DT, R, K, RY>;
    if (!fused3d_multi_ok(P, K) || passes < 1) return cudaErrorNotSupported;
    F3MpParams<C> p;
    f3_fill_common(P, p, G::W, G::H, G::WY, G::HY);
    p.src0 = src0;
    p.dst_even = dst_even;
    p.dst_odd = dst_odd;
    p.passes = passes;
    const int64_t nx = P.n[2], ny = P.n[1], nz = P.n[0];
    const bool al = ((uintptr_t)src0 % 16 == 0) && ((uintptr_t)dst_even % 16 == 0) && ((uintptr_t)dst_odd % 16 == 0);
    p.vec_ok = (nx % G::V == 0) && al;
    bool tma = P.bkind == STENCIL_DIRICHLET && ((nx * (int64_t)sizeof(S)) % 16 == 0) && al;
    CUtensorMap maps[3];
    memset(maps, 0, sizeof(maps));
    if (tma) {
        const int64_t dims[3] = {nx, ny, nz};
        const uint32_t box[3] = {(uint32_t)G::W, (uint32_t)G::WY, 1u};
        const void *bases[3] = {src0, dst_even, dst_odd};
        for (int i = 0; i < 3 && tma; ++i) tma = make_tmap(&maps[i], DT, 3, dims, box, bases[i]);
    }
    if (tma) f3_fill_common(P, p, G::W, f3_hx(R * K, G::W, G::AL), G::WY, G::HY);
    if (!tma) p.vec_ok = p.vec_ok && ((nx * (int64_t)sizeof(S)) % 16 == 0);
    auto kern = tma ? fused3d_mp_kernel<DT, R, PAT, K, RY, PROD3_TMA>
                    : fused3d_mp_kernel<DT, R, PAT, K, RY, PROD3_CPASYNC>;
    const int smem = G::SMEM;
    static bool attr_done[2] = {false, false};
    if (!attr_done[tma ? 0 : 1]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_done[tma ? 0 : 1] = true;
    }
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, G::THREADS, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    const int64_t txy = (int64_t)p.ax.T * p.ay.T;
    const int64_t slots = (int64_t)P.sm_count * bps;
    const int64_t lz = f3_lz(nz, txy, slots, R * K, P.tile_rows);
    const int64_t chunks = (nz + lz - 1) / lz;
    const int64_t tiles = txy * chunks;
    if (tiles >= (1ll << 28) || tiles * passes >= (1ll << 62)) return cudaErrorNotSupported;
    p.chunks = (int)chunks;
    p.Lz = (int)lz;
    p.tiles = (int)tiles;
    e = ensure_mp_state(P, tiles, st);
    if (e != cudaSuccess) return e;
    p.ctl = static_cast<MpCtl *>(P.d_mp);
    p.done = reinterpret_cast<int *>(static_cast<char *>(P.d_mp) + sizeof(MpCtl));
    const int64_t jobs = tiles * passes;
    const int64_t grid = jobs < slots ? jobs : slots;
    kern<<<(unsigned)grid, G::THREADS, smem, st>>>(maps[0], maps[1], maps[2], p);
    return cudaGetLastError();
}

// Largest K instantiated for (dtype, r, pattern): bounded by the registers
// that hold 2r partial planes per level (128 per thread at 512 threads); the
// boxes of radius 2 and 3 have none (they run the plain sweep).
template <int DT> constexpr int f3_kmax(int r, int pat) {
    return pat == STENCIL_BOX && r > 1 ? 0 : r == 1 ? 4 : r == 2 ? 2 : 1;
}

template <int DT, int R, int PAT>
cudaError_t launch_f3mp_k(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                          cudaStream_t st) {
    constexpr int KM = f3_kmax<DT>(R, PAT);
    switch (k) {
        case 1: if constexpr (KM >= 1) return launch_f3mp_t<DT, R, PAT, 1>(P, src0, de, dof, passes, st); break;
        case 2: if constexpr (KM >= 2) return launch_f3mp_t<DT, R, PAT, 2>(P, src0, de, dof, passes, st); break;
        case 3: if constexpr (KM >= 3) return launch_f3mp_t<DT, R, PAT, 3>(P, src0, de, dof, passes, st); break;
        case 4: if constexpr (KM >= 4) return launch_f3mp_t<DT, R, PAT, 4>(P, src0, de, dof, passes, st); break;
    }
    return cudaErrorInvalidValue;
}

// one radius, both patterns (radius 1 in k_fused3d_mp_<dtype>.cu, radii 2 and
// 3 in k_fused3d_mp_<dtype>_r23.cu: the build compiles them in parallel)
template <int DT, int R>
cudaError_t launch_f3mp_r(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                          cudaStream_t st) {
    return P.pattern == STENCIL_BOX ? launch_f3mp_k<DT, R, STENCIL_BOX>(P, src0, de, dof, k, passes, st)
                                    : launch_f3mp_k<DT, R, STENCIL_STAR>(P, src0, de, dof, k, passes, st);
}

template <int DT>
cudaError_t launch_f3mp_dt(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                           cudaStream_t st) {
    if (P.r == 1) return launch_f3mp_r<DT, 1>(P, src0, de, dof, k, passes, st);
    if (P.r == 2) return launch_f3mp_r<DT, 2>(P, src0, de, dof, k, passes, st);
    if (P.r == 3) return launch_f3mp_r<DT, 3>(P, src0, de, dof, k, passes, st);
    return cudaErrorInvalidValue;
}

template <int DT, int R, int PAT>
cudaError_t launch_f3_k(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    constexpr int KM = f3_kmax<DT>(R, PAT);
    switch (k) {
        case 1: if constexpr (KM >= 1) return launch_f3_t<DT, R, PAT, 1>(P, src, dst, st); break;
        case 2: if constexpr (KM >= 2) return launch_f3_t<DT, R, PAT, 2>(P, src, dst, st); break;
        case 3: if constexpr (KM >= 3) return launch_f3_t<DT, R, PAT, 3>(P, src, dst, st); break;
        case 4: if constexpr (KM >= 4) return launch_f3_t<DT, R, PAT, 4>(P, src, dst, st); break;
    }
    return cudaErrorInvalidValue;
}

template <int DT, int R>
cudaError_t launch_f3_r(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return P.pattern == STENCIL_BOX ? launch_f3_k<DT, R, STENCIL_BOX>(P, src, dst, k, st)
                                    : launch_f3_k<DT, R, STENCIL_STAR>(P, src, dst, k, st);
}

template <int DT>
cudaError_t launch_f3_dt(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    if (P.r == 1) return launch_f3_r<DT, 1>(P, src, dst, k, st);
    if (P.r == 2) return launch_f3_r<DT, 2>(P, src, dst, k, st);
    if (P.r == 3) return launch_f3_r<DT, 3>(P, src, dst, k, st);
    return cudaErrorInvalidValue;
}

// The pass of k <= 4 steps (radius 1) keeping every level: level l of
// src into lv[l - 1], l = 1 .. k (the adjoint's recompute of a segment).
template <int DT, int PAT>
cudaError_t launch_f3_all_k(const stencil_plan_s &P, const void *src, void *const *lv, int k, cudaStream_t st) {
    switch (k) {
        case 1: return launch_f3_t<DT, 1, PAT, 1, true>(P, src, lv[0], st, lv);
        case 2: return launch_f3_t<DT, 1, PAT, 2, true>(P, src, lv[1], st, lv);
        case 3: return launch_f3_t<DT, 1, PAT, 3, true>(P, src, lv[2], st, lv);
        case 4: return launch_f3_t<DT, 1, PAT, 4, true>(P, src, lv[3], st, lv);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sg
