// k_fused2d.cuh -- 2D Jacobi sweep with K time steps fused per pass.
//
// GPU counterpart of the paper's time-loop unroll-and-jam (Section 3.3,
// Algorithm 1).  There, vector sets stream along the grid and each is
// advanced k time levels before it is stored, the older levels kept in
// registers ("vrl") so that Jacobi semantics hold.  Here one warp streams the
// rows of a column band: every incoming row at level s contributes to 2r
// partial rows of level s+1 held in registers; the row that receives its last
// contribution is complete, is emitted as the incoming row of level s+1, and
// after K levels it is stored.  Each value is read from HBM once and written
// once per pass, so the bytes per point update drop by K.
//
//   lanes     32 lanes x V contiguous elements = a W-wide window; x-neighbours
//             across lanes come from warp shuffles (the analogue of the
//             paper's Assemble, Section 3.2); the window's outer H >= rK
//             columns are halo, recomputed redundantly (overlapped tiling);
//   rows      a job covers Ly output rows and reads rK halo rows each side;
//   input     PROD_TMA: lane 0 streams 4-row x W tiles by TMA
//             (cp.async.bulk.tensor) into a 4-stage shared-memory ring per
//             warp, completion tracked by mbarriers (bounded waits; a timeout
//             sets the status word).  Out-of-range rows/columns are
//             zero-filled by TMA and then replaced by the Dirichlet value.
//             PROD_REG: each lane loads its own V elements of the row four
//             rows ahead into registers, wrapping indices (periodic grids and
//             rows that are not 16-byte aligned);
//   boundary  Dirichlet cells outside the domain are reset to the boundary
//             value at every level (they are never computed);
//   order     each output is one multiply then FMAs over the offsets in
//             lexicographic (o_y, o_x) order, the same order as the plain
//             kernel, so every K gives bit-identical FP32/FP64 results.
#pragma once

#include "common.cuh"
#include "plan.h"

namespace sg {

constexpr int F2_NW = 4;       // default warps per CTA (independent jobs); 1..F2_MAXNW at launch
constexpr int F2_MAXNW = 8;
constexpr int F2_ROWS = 4;     // rows per TMA stage
constexpr int F2_STAGES = 4;   // TMA ring depth per warp (3 stages = 12 rows in flight)
constexpr int F2_PREF = 4;     // rows prefetched in registers (PROD_REG)
constexpr int F2_U = 4;        // step unroll: multiple of 2R (R <= 2) and of F2_PREF
enum { PROD_TMA = 0, PROD_REG = 1 };

template <int DT, int R, int K> struct F2Geo {
    using S = typename Traits<DT>::S;
    static constexpr int V = Traits<DT>::V;
    static constexpr int W = 32 * V;
    static constexpr int AL = max_c(align_elems<DT>(), V);
    static constexpr int H = round_up_c(R * K, AL);
    static constexpr int BW = W - 2 * H;
    static constexpr int STAGE_ELEMS = F2_ROWS * W;
    static constexpr int STAGE_BYTES = STAGE_ELEMS * (int)sizeof(S);
    static constexpr int WARP_SMEM = F2_STAGES * STAGE_BYTES;
    static constexpr int WARP_BYTES = WARP_SMEM + F2_STAGES * 8;   // a warp's stages and barriers
    static_assert(BW >= V, "fusion depth too large for the window");
};

template <typename C> struct F2Params {
    GridGeom<C> g;     // n0 = 1, n1 = ny, n2 = nx
    const void *src;
    void *dst;
    int64_t jobs;
    int64_t bands;
    int64_t Ly;
    int vec_ok;        // rows and both base pointers allow V-wide vector access
    int *status;
    JobCtl *ctl;       // job tickets (left at zero by the launch's last warp)
    C w[49];           // evaluation order; up to the r = 3 box
};

// Control block of a persistent multi-pass launch: the item ticket, the
// abort flag raised when a dependency wait gives up, and the exit count.
struct MpCtl {
    unsigned long long ticket;
    int abort;
    unsigned exited;
};

static_assert(sizeof(MpCtl) == kMpCtlBytes, "control block layout");

template <typename C> struct F2MpParams {
    GridGeom<C> g;     // n0 = 1, n1 = ny, n2 = nx
    const void *src0;  // input of pass 0
    void *dst_even;    // output of the passes p with (passes - 1 - p) even (includes the last)
    void *dst_odd;     // output of the other passes
    int passes;
    int bands, chunks, Ly;
    int vec_ok;
    int *status;
    MpCtl *ctl;        // ticket, abort flag, exit count
    int *done;         // [tiles]: passes each tile has finished
    int tiles;         // (all left at zero by the launch's last warp)
    C w[49];
};

// ------------------------------------------------------------ memory helpers
template <bool COH, typename T> __device__ __forceinline__ T ldx(const T *p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// V contiguous storage elements (16 or 8 bytes) -> arithmetic values
template <int DT, bool COH>
__device__ __forceinline__ void ldvec(const typename Traits<DT>::S *p, typename Traits<DT>::C *out) {
    using S = typename Traits<DT>::S;
    constexpr int V = Traits<DT>::V;
    constexpr int BYTES = V * (int)sizeof(S);
    if constexpr (BYTES == 16) {
        uint4 v = ldx<COH>(reinterpret_cast<const uint4 *>(p));
        const S *s = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = to_c(s[i]);
    } else {
        static_assert(BYTES == 8, "vector width");
        uint2 v = ldx<COH>(reinterpret_cast<const uint2 *>(p));
        const S *s = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = to_c(s[i]);
    }
}

template <int DT>
__device__ __forceinline__ void stvec(typename Traits<DT>::S *p, const typename Traits<DT>::C *in) {
    using S = typename Traits<DT>::S;
    constexpr int V = Traits<DT>::V;
    constexpr int BYTES = V * (int)sizeof(S);
    S tmp[V];
#pragma unroll
    for (int i = 0; i < V; ++i) tmp[i] = from_c<S>(in[i]);
    if constexpr (BYTES == 16) *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(tmp);
    else *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(tmp);
}

template <int DT>
__device__ __forceinline__ void ldsvec(const typename Traits<DT>::S *p, typename Traits<DT>::C *out) {
    using S = typename Traits<DT>::S;
    constexpr int V = Traits<DT>::V;
    constexpr int BYTES = V * (int)sizeof(S);
    if constexpr (BYTES == 16) {
        uint4 v = *reinterpret_cast<const uint4 *>(p);
        const S *s = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = to_c(s[i]);
    } else {
        uint2 v = *reinterpret_cast<const uint2 *>(p);
        const S *s = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = to_c(s[i]);
    }
}

// V values returned by value (registers) from an out-of-line function
template <typename C, int V> struct LaneVals {
    C v[V];
};

// The rare cases of load_row_reg, kept out of line so that the unrolled job
// loops hold only the vector path: a row wrapped more than once, and lanes
// whose V elements straddle the row's end or cannot be read as one vector.
template <int DT, bool COH>
__device__ __noinline__ LaneVals<typename Traits<DT>::C, Traits<DT>::V> load_row_edge(
    const typename Traits<DT>::S *__restrict__ src, int64_t nx, int64_t ny, bool periodic,
    typename Traits<DT>::C bval, int64_t y, int64_t xl) {
    constexpr int V = Traits<DT>::V;
    LaneVals<typename Traits<DT>::C, V> r;
    y = wrap_idx(y, ny);
    const typename Traits<DT>::S *row = src + y * nx;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int64_t x = xl + v;
        if (x >= 0 && x < nx) r.v[v] = to_c(ldx<COH>(row + x));
        else if (periodic) r.v[v] = to_c(ldx<COH>(row + wrap_idx(x, nx)));
        else r.v[v] = bval;
    }
    return r;
}

// One lane's V elements of virtual row y, columns xl..xl+V-1, through the
// boundary rule (PROD_REG input path).
template <int DT, bool COH>
__device__ __forceinline__ void load_row_reg(const typename Traits<DT>::S *__restrict__ src, int64_t nx, int64_t ny,
                                             bool periodic, typename Traits<DT>::C bval, int64_t y, int64_t xl,
                                             bool vec_ok, typename Traits<DT>::C *out) {
    constexpr int V = Traits<DT>::V;
    if (y < 0 || y >= ny) {
        if (!periodic) {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = bval;
            return;
        }
        y = y < 0 ? y + ny : y - ny;
    }
    // a lane's V elements outside a periodic row, wrapped by one extent, are
    // still one vector when the row length is a multiple of V
    int64_t xs = xl;
    bool xin = xl >= 0 && xl + V <= nx;
    if (!xin && periodic) {
        xs = xl < 0 ? xl + nx : xl - nx;
        xin = xs >= 0 && xs + V <= nx;
    }
    if (vec_ok && xin && y >= 0 && y < ny) {
        ldvec<DT, COH>(src + y * nx + xs, out);
    } else {
        const LaneVals<typename Traits<DT>::C, V> r = load_row_edge<DT, COH>(src, nx, ny, periodic, bval, y, xl);
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = r.v[v];
    }
}

// ------------------------------------------------------------- one job
// Advances the rows [yo0, yo1) x columns [xo0, xo0 + BW) of one grid by K
// steps.  Returns false if a bounded wait gave up (caller records status).
template <int DT, int R, int PAT, int K, int PROD, bool COH, bool MASK>
__device__ __forceinline__ bool fused2d_job(const CUtensorMap *tmap, const typename Traits<DT>::S *__restrict__ src,
                                            typename Traits<DT>::S *__restrict__ dst, int64_t nx, int64_t ny,
                                            bool dir, typename Traits<DT>::C bval, const typename Traits<DT>::C *wr,
                                            int64_t xo0, int64_t yo0, int64_t yo1, bool vec_ok,
                                            typename Traits<DT>::S *stg, uint64_t *bars, uint32_t &gst, int lane) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F2Geo<DT, R, K>;
    using Sh = Shape<2, R, PAT>;
    constexpr int V = G::V, W = G::W, H = G::H, BW = G::BW, NS = 2 * R;
    // step unroll: the partial-row slots repeat every 2R rows and the register
    // prefetch ring (PROD_REG) every F2_PREF rows: U = lcm(2R, F2_PREF) (4 for
    // r <= 2, 12 for r = 3).  The position within a TMA stage of F2_ROWS rows
    // is a run-time index, so box stencils fed by TMA unroll only U = 2R: half
    // the code of their (large) loop body for r = 1, whose instruction fetch
    // limited it (2D9P +6 %); the star keeps the longer unroll (2D5P -3 % with
    // the short one)
    constexpr int U = PROD == PROD_TMA && PAT == STENCIL_BOX ? NS : lcm_c(NS, F2_PREF);
    static_assert(U % NS == 0 && (PROD == PROD_TMA || U % F2_PREF == 0), "unroll");
    static_assert((F2_ROWS & (F2_ROWS - 1)) == 0, "stage rows: a power of two");
    constexpr uint32_t FULLM = (1u << V) - 1u;

    // row indices fit in 32 bits (checked by the launcher)
    const int64_t xw0 = xo0 - H;
    const int64_t xl = xw0 + (int64_t)lane * V;
    const int ny32 = (int)ny;
    const int yi0 = (int)yo0 - R * K;
    const int yo0i = (int)yo0, yo1i = (int)yo1;
    const int nsteps = (yo1i - yo0i) + 2 * R * K;
    const int nsp = round_up_c(nsteps, U);
    uint32_t cmask = 0;
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (xl + v >= 0 && xl + v < nx) cmask |= 1u << v;
    const bool need_cmask = MASK && __any_sync(0xffffffffu, cmask != FULLM);
    bool keep[V];
#pragma unroll
    for (int v = 0; v < V; ++v) keep[v] = (cmask >> v) & 1u;
    const bool lane_out = (lane * V >= H) && (lane * V < H + BW);

    int nst = 0;
    C ring[F2_PREF][V];
    if constexpr (PROD == PROD_TMA) {
        nst = (nsp + F2_ROWS - 1) / F2_ROWS;
        __syncwarp();   // every lane is done with the previous job's stages
        if (lane == 0) {
            fence_proxy_async_smem();
            const int pre = nst < F2_STAGES ? nst : F2_STAGES;
            for (int q = 0; q < pre; ++q) {
                const uint32_t g = gst + q, slot = g % F2_STAGES;
                mbar_arrive_expect_tx(&bars[slot], G::STAGE_BYTES);
                tma_load_2d(stg + slot * G::STAGE_ELEMS, tmap, &bars[slot], (int)xw0, (int)(yi0 + q * F2_ROWS));
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < F2_PREF; ++q)
            load_row_reg<DT, COH>(src, nx, ny, !dir, bval, yi0 + q, xl, vec_ok, ring[q]);
    }

    C P[K][NS][V];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int m = 0; m < NS; ++m)
#pragma unroll
            for (int v = 0; v < V; ++v) P[s][m][v] = C(0);

    // stage ring position: slot and phase parity advance once per stage
    uint32_t slot = gst % F2_STAGES, par = (gst / F2_STAGES) & 1u;
    int q = 0;                                   // stage index within the job
    const S *srow = stg + slot * G::STAGE_ELEMS + lane * V;
    for (int i0 = 0; i0 < nsp; i0 += U) {
#pragma unroll
        for (int ph = 0; ph < U; ++ph) {
        const int rr = (i0 + ph) & (F2_ROWS - 1);   // row within the TMA stage
        if constexpr (PROD == PROD_TMA) {
            if (rr == 0) {
                const bool ok = mbar_wait_bounded(&bars[slot], par);
                if (__any_sync(0xffffffffu, !ok)) {
                    // give up: wait (bounded, about ten seconds per stage) for
                    // this warp's copies in flight before its shared memory can
                    // be left; the caller records the timeout either way
                    if (lane == 0)
                        for (int qq = q; qq < nst && qq < q + F2_STAGES; ++qq) {
                            const uint32_t gg = gst + qq;
                            if (!mbar_drain(&bars[gg % F2_STAGES], (gg / F2_STAGES) & 1u)) break;
                        }
                    __syncwarp();
                    return false;
                }
                srow = stg + slot * G::STAGE_ELEMS + lane * V;
            }
        }
        {
            const int i = i0 + ph;
            const int yin = yi0 + i;
            C cur[V];
            if constexpr (PROD == PROD_TMA) {
                ldsvec<DT>(srow + rr * W, cur);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) cur[v] = ring[ph % F2_PREF][v];
                load_row_reg<DT, COH>(src, nx, ny, !dir, bval, (int64_t)yin + F2_PREF, xl, vec_ok, ring[ph % F2_PREF]);
            }
            if constexpr (MASK) {
                if ((unsigned)yin >= (unsigned)ny32) {
#pragma unroll
                    for (int v = 0; v < V; ++v) cur[v] = bval;
                } else if (need_cmask) {
#pragma unroll
                    for (int v = 0; v < V; ++v) cur[v] = keep[v] ? cur[v] : bval;
                }
            }
#pragma unroll
            for (int s = 0; s < K; ++s) {
                // cur: level-s row J = yin - sR.  Partial rows of level s+1:
                // Y = J - R + m sits in slot (ph + m) % NS.
                C ext[V + 2 * R];
#pragma unroll
                for (int v = 0; v < V; ++v) ext[R + v] = cur[v];
                // the value qq + 1 columns beyond the lane's edge sits in the
                // lane qq / V + 1 positions away
#pragma unroll
                for (int qq = 0; qq < R; ++qq) {
                    ext[R - 1 - qq] = __shfl_up_sync(0xffffffffu, cur[V - 1 - qq % V], qq / V + 1);
                    ext[R + V + qq] = __shfl_down_sync(0xffffffffu, cur[qq % V], qq / V + 1);
                }
                C emit[V];
                const int s0 = ph % NS;
                // complete Y = J - R with its o_y = +R terms
#pragma unroll
                for (int v = 0; v < V; ++v) emit[v] = P[s][s0][v];
#pragma unroll
                for (int ox = -R; ox <= R; ++ox) {
                    if (!Sh::inc(0, R, ox)) continue;
                    row_fma_s<C, V>(wr[Sh::widx(0, R, ox)], &ext[R + ox], emit);
                }
                // rows Y = J - R + m (0 < m < 2R) take their o_y = R - m terms
#pragma unroll
                for (int m = 1; m < NS; ++m) {
                    const int oy = R - m;
                    const int sl = (ph + m) % NS;
#pragma unroll
                    for (int ox = -R; ox <= R; ++ox) {
                        if (!Sh::inc(0, oy, ox)) continue;
                        row_fma_s<C, V>(wr[Sh::widx(0, oy, ox)], &ext[R + ox], P[s][sl]);
                    }
                }
                // start Y = J + R with its o_y = -R terms (first term: multiply)
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
                // emitted row Y = yin - (s+1)R: Dirichlet cells keep the boundary value
                if constexpr (MASK) {
                    const int ye = yin - (s + 1) * R;
                    if ((unsigned)ye >= (unsigned)ny32) {
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
            // level-K row
            const int yout = yin - K * R;
            if (yout >= yo0i && yout < yo1i && lane_out) {
                S *rowp = dst + (int64_t)yout * nx;
                if (vec_ok && xl + V <= nx) {
                    stvec<DT>(rowp + xl, cur);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (xl + v < nx) rowp[xl + v] = from_c<S>(cur[v]);
                }
            }
        }
        if constexpr (PROD == PROD_TMA) {
            if (rr == F2_ROWS - 1) {
                // stage consumed by every lane: refill it with the stage S ahead
                __syncwarp();
                if (lane == 0 && q + F2_STAGES < nst) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&bars[slot], G::STAGE_BYTES);
                    tma_load_2d(stg + slot * G::STAGE_ELEMS, tmap, &bars[slot], (int)xw0,
                                yi0 + (q + F2_STAGES) * F2_ROWS);
                }
                ++q;
                if (++slot == F2_STAGES) { slot = 0; par ^= 1u; }
            }
        }
        }
    }
    gst += (uint32_t)nst;
    return true;
}

// Resident 4-warp CTAs per SM the register allocation must allow.  Up to the
// partial-row registers of r = 1, k = 8 the measured table by fusion depth;
// beyond it, what 2r k V partial values (plus about 96 other registers) per
// thread leave room for; radius 3 (49-term box, 12-step unroll) gets 168 or
// 255 registers.
template <int DT, int R, int K> constexpr int f2_min_blocks() {
    constexpr int pr = K * 2 * R * Traits<DT>::V * (int)(sizeof(typename Traits<DT>::C) / 4);
    constexpr int regs = round_up_c(pr + 96, 8);
    return R == 3 ? (pr <= 48 ? 3 : 2)
         : pr <= 64 ? (K <= 3 ? 6 : K <= 5 ? 5 : K <= 6 ? 4 : 3)
                    : (65536 / (F2_NW * 32 * regs) < 2 ? 2 : 65536 / (F2_NW * 32 * regs));
}

// the per-thread register cap those resident CTAs imply (the same cap a
// 4-warp launch bound would give), so that the kernels can be launched with
// any block size of 1..F2_MAXNW warps
template <int DT, int R, int K> constexpr int f2_regcap() {
    return (65536 / (F2_NW * 32 * f2_min_blocks<DT, R, K>())) / 8 * 8 > 255
               ? 255
               : (65536 / (F2_NW * 32 * f2_min_blocks<DT, R, K>())) / 8 * 8;
}

template <int DT, int R, int PAT, int K, int PROD>
__global__ void __launch_bounds__(F2_MAXNW * 32) __maxnreg__((f2_regcap<DT, R, K>()))
    fused2d_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ F2Params<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F2Geo<DT, R, K>;
    using Sh = Shape<2, R, PAT>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S *stg = reinterpret_cast<S *>(smem + warp * G::WARP_SMEM);
    const int nw = (int)(blockDim.x >> 5);   // warps in this CTA (the launch's block size)
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + nw * G::WARP_SMEM) + warp * F2_STAGES;
    if constexpr (PROD == PROD_TMA) {
        if (lane == 0) {
            for (int s = 0; s < F2_STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
            prefetch_tmap(&tmap);
        }
        __syncwarp();
    }
    const C *wr = p.w;   // parameter space: FMAs can read the weights as constant operands
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    uint32_t gst = 0;
    // jobs are taken dynamically, so faster SMs take more; the first and last
    // row chunks (Dirichlet edges, the slower jobs) come first
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&p.ctl->ticket, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)p.jobs) break;
        const int64_t band = (int64_t)(t % p.bands), tc = (int64_t)(t / p.bands);
        const int64_t nch = p.jobs / p.bands;
        const int64_t chunk = nch < 2 ? tc : (tc == 0 ? 0 : tc == 1 ? nch - 1 : tc - 1);
        const int64_t yo0 = chunk * p.Ly;
        const int64_t yo1 = yo0 + p.Ly < p.g.n1 ? yo0 + p.Ly : p.g.n1;
        const int64_t xo0 = band * G::BW;
        // jobs whose window and rows lie inside the domain never see a
        // Dirichlet cell: they run without any masking code
        const bool interior = !dir || (xo0 - G::H >= 0 && xo0 - G::H + G::W <= p.g.n2 && yo0 - R * K >= 0 &&
                                       yo1 + R * K <= p.g.n1);
        const bool ok = interior
            ? fused2d_job<DT, R, PAT, K, PROD, false, false>(&tmap, static_cast<const S *>(p.src), static_cast<S *>(p.dst),
                                                            p.g.n2, p.g.n1, dir, p.g.bval, wr, xo0, yo0, yo1,
                                                            p.vec_ok != 0, stg, bars, gst, lane)
            : fused2d_job<DT, R, PAT, K, PROD, false, true>(&tmap, static_cast<const S *>(p.src), static_cast<S *>(p.dst),
                                                           p.g.n2, p.g.n1, dir, p.g.bval, wr, xo0, yo0, yo1,
                                                           p.vec_ok != 0, stg, bars, gst, lane);
        if (!ok) {
            if (lane == 0) record_status(p.status, kStatusTimeout);
            break;
        }
    }
    __syncwarp();
    if (lane == 0 && worker_exit_is_last(&p.ctl->exited, gridDim.x * nw)) {
        p.ctl->ticket = 0ull;
        p.ctl->exited = 0u;
    }
}

// All `passes` passes of stencil_run (K steps each) in one persistent launch.
// Warps take (pass, tile) items from one ticket, pass-major and row-major
// within a pass.  Before an item of pass p starts, every tile whose output
// meets its input window must have finished pass p - 1: those are the tiles
// whose outputs it reads and, since the relation is symmetric, the tiles whose
// inputs (the buffer pass p + 1 ... reuses) its output overwrites -- so each
// item reads finished data and never overwrites data still being read.
// Every dependency has an earlier ticket, held by a running warp, so the
// waits end; they are still bounded (about one second), and a wait that gives
// up raises the abort flag, stops every warp and records STENCIL_ERR_TIMEOUT.
// The per-pass tail of the one-launch-per-pass form (warps idle while the
// last jobs of a pass finish) then occurs once per run.
template <int DT, int R, int PAT, int K, int PROD>
__global__ void __launch_bounds__(F2_MAXNW * 32) __maxnreg__((f2_regcap<DT, R, K>()))
    fused2d_mp_kernel(const __grid_constant__ CUtensorMap tm_src0, const __grid_constant__ CUtensorMap tm_even,
                      const __grid_constant__ CUtensorMap tm_odd, const __grid_constant__ F2MpParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F2Geo<DT, R, K>;
    constexpr bool COH = PROD == PROD_REG;   // register loads must bypass L1: other SMs wrote the data
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S *stg = reinterpret_cast<S *>(smem + warp * G::WARP_SMEM);
    const int nw = (int)(blockDim.x >> 5);   // warps in this CTA (the launch's block size)
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + nw * G::WARP_SMEM) + warp * F2_STAGES;
    if constexpr (PROD == PROD_TMA) {
        if (lane == 0) {
            for (int s = 0; s < F2_STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
            prefetch_tmap(&tm_src0);
            prefetch_tmap(&tm_even);
            prefetch_tmap(&tm_odd);
        }
        __syncwarp();
    }
    MpCtl *ctl = p.ctl;
    int *done = p.done;
    const C *wr = p.w;
    const bool dir = p.g.bkind == STENCIL_DIRICHLET;
    const int nx = (int)p.g.n2, ny = (int)p.g.n1;
    const int jobs = p.bands * p.chunks;
    const unsigned long long items = (unsigned long long)jobs * (unsigned)p.passes;
    uint32_t gst = 0;
    // the next ticket and the abort flag are fetched one job ahead, so that
    // their latency overlaps the current job
    unsigned long long t_next = 0;
    int ab_next = 0;
    if (lane == 0) t_next = atomicAdd(&ctl->ticket, 1ull);
    for (;;) {
        const unsigned long long t = __shfl_sync(0xffffffffu, t_next, 0);
        const int ab = __shfl_sync(0xffffffffu, ab_next, 0);
        if (t >= items || ab) break;
        if (lane == 0) {
            t_next = atomicAdd(&ctl->ticket, 1ull);
            ab_next = ld_relaxed(&ctl->abort);
        }
        const int pass = (int)(t / (unsigned)jobs), j = (int)(t % (unsigned)jobs);
        const int chunk = j / p.bands, band = j - chunk * p.bands;
        const int yo0 = chunk * p.Ly;
        const int yo1 = yo0 + p.Ly < ny ? yo0 + p.Ly : ny;
        const int xo0 = band * G::BW;
        if (pass > 0) {
            const int xe = xo0 + G::BW < nx ? xo0 + G::BW : nx;
            const TileSpan sb = tile_span(xo0 - G::H, xe + G::H, nx, G::BW, !dir);
            const TileSpan sc = tile_span(yo0 - R * K, yo1 + R * K, ny, p.Ly, !dir);
            const int nb = sb.count(), nd = nb * sc.count();
            bool ok = true;
            for (int e = lane; e < nd; e += 32) {
                const int b2 = sb.at(e % nb), c2 = sc.at(e / nb);
                ok = ok && wait_counter(&done[c2 * p.bands + b2], pass, &ctl->abort);
            }
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    atomicExch(&ctl->abort, 1);
                    record_status(p.status, kStatusTimeout);
                }
                break;
            }
            // every lane's acquire precedes every lane's reads; TMA reads
            // (async proxy) also need the proxy fence
            __syncwarp();
            if constexpr (PROD == PROD_TMA) {
                if (lane == 0) fence_proxy_async_global();
            }
        }
        const bool from_even = ((p.passes - pass) & 1) == 0;   // pass - 1 wrote dst_even
        const S *src = static_cast<const S *>(pass == 0 ? p.src0 : from_even ? p.dst_even : p.dst_odd);
        const CUtensorMap *tm = pass == 0 ? &tm_src0 : from_even ? &tm_even : &tm_odd;
        S *dst = static_cast<S *>(((p.passes - 1 - pass) & 1) == 0 ? p.dst_even : p.dst_odd);
        const bool interior = !dir || (xo0 - G::H >= 0 && xo0 - G::H + G::W <= nx && yo0 - R * K >= 0 &&
                                       yo1 + R * K <= ny);
        const bool ok = interior
            ? fused2d_job<DT, R, PAT, K, PROD, COH, false>(tm, src, dst, nx, ny, dir, p.g.bval, wr, xo0, yo0, yo1,
                                                          p.vec_ok != 0, stg, bars, gst, lane)
            : fused2d_job<DT, R, PAT, K, PROD, COH, true>(tm, src, dst, nx, ny, dir, p.g.bval, wr, xo0, yo0, yo1,
                                                         p.vec_ok != 0, stg, bars, gst, lane);
        if (!ok) {
            if (lane == 0) {
                atomicExch(&ctl->abort, 1);
                record_status(p.status, kStatusTimeout);
            }
            break;
        }
        // publish: every lane's stores, then (release) the tile's pass count
        __syncwarp();
        if (lane == 0) {
            if constexpr (PROD == PROD_TMA) fence_proxy_async_global();
            red_release_add(&done[j], 1);
        }
    }
    // the last warp out leaves the counters at zero for the next launch
    __syncwarp();
    int last = 0;
    if (lane == 0) last = worker_exit_is_last(&ctl->exited, gridDim.x * nw);
    if (__shfl_sync(0xffffffffu, last, 0)) {
        for (int i = lane; i < p.tiles; i += 32) done[i] = 0;
        if (lane == 0) {
            ctl->ticket = 0ull;
            ctl->abort = 0;
            ctl->exited = 0u;
        }
    }
}

// ------------------------------------------------------------------ host side
template <typename C> C conv_w(double w) {
    if constexpr (sizeof(C) == 4 && C(-1) > C(0)) return (C)(uint32_t)(int64_t)w;
    else return (C)w;
}

// Column bands of BW and row chunks of Ly: `rows` high if set, else about
// `per_slot` jobs per resident warp; chunks at least max(4 r k, 16) rows.
struct F2Tiling {
    int64_t bands, chunks, Ly;
};
inline F2Tiling f2_tiling(int64_t nx, int64_t ny, int bw, int rk, int64_t slots, int per_slot, int rows) {
    F2Tiling t;
    t.bands = (nx + bw - 1) / bw;
    const int64_t min_ly = 4 * rk > 16 ? 4 * rk : 16;
    if (rows > 0) {
        t.Ly = rows > min_ly ? rows : min_ly;
        if (t.Ly > ny) t.Ly = ny;
    } else {
        int64_t chunks = per_slot * slots / t.bands;
        if (chunks < 1) chunks = 1;
        const int64_t max_chunks = ny / min_ly > 1 ? ny / min_ly : 1;
        if (chunks > max_chunks) chunks = max_chunks;
        t.Ly = (ny + chunks - 1) / chunks;
    }
    t.chunks = (ny + t.Ly - 1) / t.Ly;
    return t;
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_f2_t(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F2Geo<DT, R, K>;
    F2Params<C> p;
    p.g.n0 = 1;
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.src = src;
    p.dst = dst;
    p.status = P.d_status;
    p.ctl = static_cast<JobCtl *>(P.d_ctr);
    if (P.np > (int)(sizeof(p.w) / sizeof(p.w[0]))) return cudaErrorInvalidValue;   // weights fit the parameter block
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    const int64_t nx = P.n[2], ny = P.n[1];
    if (ny + 4 * R * K + 64 >= (1ll << 31)) return cudaErrorNotSupported;   // rows are 32-bit in the kernel
    p.vec_ok = (nx % G::V == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
    bool tma = P.bkind == STENCIL_DIRICHLET && ((nx * (int64_t)sizeof(S)) % 16 == 0) && ((uintptr_t)src % 16 == 0) &&
               nx < (1ll << 31) && ny < (1ll << 31);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (tma) {
        const int64_t dims[2] = {nx, ny};
        const uint32_t box[2] = {(uint32_t)G::W, (uint32_t)F2_ROWS};
        tma = make_tmap(&map, DT, 2, dims, box, src);
    }
    auto kern = tma ? fused2d_kernel<DT, R, PAT, K, PROD_TMA> : fused2d_kernel<DT, R, PAT, K, PROD_REG>;
    const int nw = P.block_warps > 0 ? P.block_warps : F2_NW;
    const int smem = tma ? nw * G::WARP_BYTES : 0;
    static bool attr_done[2] = {false, false};
    if (!attr_done[tma ? 0 : 1]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tma ? F2_MAXNW * G::WARP_BYTES : 0);
        if (e != cudaSuccess) return e;
        attr_done[tma ? 0 : 1] = true;
    }
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, nw * 32, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    const F2Tiling tl = f2_tiling(nx, ny, G::BW, R * K, (int64_t)P.sm_count * bps * nw, 2, P.tile_rows);
    p.Ly = tl.Ly;
    p.bands = tl.bands;
    p.jobs = tl.bands * tl.chunks;
    int64_t grid = (p.jobs + nw - 1) / nw;
    if (grid > (int64_t)P.sm_count * bps) grid = (int64_t)P.sm_count * bps;
    kern<<<(unsigned)grid, nw * 32, smem, st>>>(map, p);
    return cudaGetLastError();
}

template <int DT, int R, int PAT, int K>
cudaError_t launch_f2mp_t(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int passes,
                          cudaStream_t st) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using G = F2Geo<DT, R, K>;
    if (!fused2d_multi_ok(P, K) || passes < 1) return cudaErrorNotSupported;
    F2MpParams<C> p;
    p.g.n0 = 1;
    p.g.n1 = P.n[1];
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.src0 = src0;
    p.dst_even = dst_even;
    p.dst_odd = dst_odd;
    p.passes = passes;
    p.status = P.d_status;
    if (P.np > (int)(sizeof(p.w) / sizeof(p.w[0]))) return cudaErrorInvalidValue;   // weights fit the parameter block
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    const int64_t nx = P.n[2], ny = P.n[1];
    const bool al = ((uintptr_t)src0 % 16 == 0) && ((uintptr_t)dst_even % 16 == 0) && ((uintptr_t)dst_odd % 16 == 0);
    p.vec_ok = (nx % G::V == 0) && al;
    bool tma = P.bkind == STENCIL_DIRICHLET && ((nx * (int64_t)sizeof(S)) % 16 == 0) && al;
    CUtensorMap maps[3];
    memset(maps, 0, sizeof(maps));
    if (tma) {
        const int64_t dims[2] = {nx, ny};
        const uint32_t box[2] = {(uint32_t)G::W, (uint32_t)F2_ROWS};
        const void *bases[3] = {src0, dst_even, dst_odd};
        for (int i = 0; i < 3 && tma; ++i) tma = make_tmap(&maps[i], DT, 2, dims, box, bases[i]);
    }
    auto kern = tma ? fused2d_mp_kernel<DT, R, PAT, K, PROD_TMA> : fused2d_mp_kernel<DT, R, PAT, K, PROD_REG>;
    const int nw = P.block_warps > 0 ? P.block_warps : F2_NW;
    const int smem = tma ? nw * G::WARP_BYTES : 0;
    static bool attr_done[2] = {false, false};
    if (!attr_done[tma ? 0 : 1]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tma ? F2_MAXNW * G::WARP_BYTES : 0);
        if (e != cudaSuccess) return e;
        attr_done[tma ? 0 : 1] = true;
    }
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, nw * 32, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    const int64_t slots = (int64_t)P.sm_count * bps * nw;
    // about three jobs per resident warp and pass: the next pass's items find
    // their dependencies finished (with one job per warp the passes would
    // run in lock step)
    const F2Tiling tl = f2_tiling(nx, ny, G::BW, R * K, slots, 3, P.tile_rows);
    if (tl.bands * tl.chunks >= (1ll << 30) / 4 || tl.bands * tl.chunks * (int64_t)passes >= (1ll << 62))
        return cudaErrorNotSupported;
    p.bands = (int)tl.bands;
    p.chunks = (int)tl.chunks;
    p.Ly = (int)tl.Ly;
    p.tiles = (int)(tl.bands * tl.chunks);
    e = ensure_mp_state(P, p.tiles, st);
    if (e != cudaSuccess) return e;
    p.ctl = static_cast<MpCtl *>(P.d_mp);
    p.done = reinterpret_cast<int *>(static_cast<char *>(P.d_mp) + sizeof(MpCtl));
    const int64_t jobs = (int64_t)p.tiles * passes;
    int64_t grid = (jobs + nw - 1) / nw;
    if (grid > (int64_t)P.sm_count * bps) grid = (int64_t)P.sm_count * bps;
    kern<<<(unsigned)grid, nw * 32, smem, st>>>(maps[0], maps[1], maps[2], p);
    return cudaGetLastError();
}

// Largest K instantiated for (dtype, r): bounded by the partial rows a lane
// keeps in registers (2r per level) and by the window's halo (W - 2H >= V).
// Depths beyond 8 are built for FP32 and int32 storage (the benchmarked and
// the bit-exact types); FP64 and the half-precision storage types stop at 8
// (radius 1), 4 (radius 2) and 2 (radius 3), which keeps the build short.
template <int DT> constexpr int f2_kmax(int r) {
    return (DT == STENCIL_F32 || DT == STENCIL_I32) ? (r == 1 ? 16 : r == 2 ? 4 : 2)
                                                    : (r == 1 ? 8 : r == 2 ? 4 : 2);
}

// Depths above 8 exist only as the persistent multi-pass kernel; a single
// pass of such a depth runs as that kernel with one pass.
constexpr int F2_PER_PASS_KMAX = 8;

// Fusion depths KLO..KHI of one radius and both patterns; each (dtype,
// radius, depth range) is instantiated in a translation unit of its own, so
// that the build compiles them in parallel.
template <int DT, int R, int K, int KHI>
cudaError_t launch_f2_kr(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    if constexpr (K > KHI || K > f2_kmax<DT>(R) || K > F2_PER_PASS_KMAX) {
        return cudaErrorInvalidValue;
    } else {
        if (k == K)
            return P.pattern == STENCIL_BOX ? launch_f2_t<DT, R, STENCIL_BOX, K>(P, src, dst, st)
                                            : launch_f2_t<DT, R, STENCIL_STAR, K>(P, src, dst, st);
        return launch_f2_kr<DT, R, K + 1, KHI>(P, src, dst, k, st);
    }
}

template <int DT, int R, int K, int KHI>
cudaError_t launch_f2mp_kr(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                           cudaStream_t st) {
    if constexpr (K > KHI || K > f2_kmax<DT>(R)) {
        return cudaErrorInvalidValue;
    } else {
        if (k == K)
            return P.pattern == STENCIL_BOX ? launch_f2mp_t<DT, R, STENCIL_BOX, K>(P, src0, de, dof, passes, st)
                                            : launch_f2mp_t<DT, R, STENCIL_STAR, K>(P, src0, de, dof, passes, st);
        return launch_f2mp_kr<DT, R, K + 1, KHI>(P, src0, de, dof, k, passes, st);
    }
}

// entry points of the instantiation units: radius 1 depths 1..8 (with the
// dispatcher), radius 1 depths 9..16, radius 2, radius 3
template <int DT, int R, int KLO, int KHI>
cudaError_t launch_f2_range(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    return launch_f2_kr<DT, R, KLO, KHI>(P, src, dst, k, st);
}
template <int DT, int R, int KLO, int KHI>
cudaError_t launch_f2mp_range(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                              cudaStream_t st) {
    return launch_f2mp_kr<DT, R, KLO, KHI>(P, src0, de, dof, k, passes, st);
}

// (depths above F2_PER_PASS_KMAX: launch_fused2d runs the persistent kernel)
template <int DT>
cudaError_t launch_f2_dt(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    if (k > F2_PER_PASS_KMAX) return cudaErrorNotSupported;
    if (P.r == 1) return launch_f2_range<DT, 1, 1, 8>(P, src, dst, k, st);
    if (P.r == 2) return launch_f2_range<DT, 2, 1, 16>(P, src, dst, k, st);
    if (P.r == 3) return launch_f2_range<DT, 3, 1, 16>(P, src, dst, k, st);
    return cudaErrorInvalidValue;
}

template <int DT>
cudaError_t launch_f2mp_dt(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                           cudaStream_t st) {
    if (P.r == 1) return k <= 8 ? launch_f2mp_range<DT, 1, 1, 8>(P, src0, de, dof, k, passes, st)
                                : launch_f2mp_range<DT, 1, 9, 16>(P, src0, de, dof, k, passes, st);
    if (P.r == 2) return launch_f2mp_range<DT, 2, 1, 16>(P, src0, de, dof, k, passes, st);
    if (P.r == 3) return launch_f2mp_range<DT, 3, 1, 16>(P, src0, de, dof, k, passes, st);
    return cudaErrorInvalidValue;
}

}  // namespace sg
