// k_fused1d.cuh -- 1D Jacobi sweep with K time steps fused per pass.
//
// The GPU form of the paper's Algorithm 1 (Section 3.3), laid along x.  A
// warp streams "vector sets" of 32 x V contiguous elements (lane l holds V
// neighbours, the analogue of one transposed vector set); for each of the K
// levels it keeps the chunk waiting for its right neighbour (VS_i) and the
// last r values of the chunk before it (vrl_i, the old values that keep the
// update Jacobi rather than Gauss-Seidel).  When chunk A arrives at level s,
// level s+1 of chunk A-1 is computed -- left neighbours from the previous
// lane or vrl, right neighbours from the next lane or the head of chunk A
// (warp shuffles: the analogue of Assemble) -- and passed on as level s+1's
// incoming chunk.  After K levels the chunk is stored: one HBM read and one
// write per point per pass.  Requires K r <= 32 V (the halo a job reads is
// one chunk on each side).
#pragma once

#include <algorithm>
#include <string>

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

constexpr int F1_NW = 4;      // warps per CTA (independent jobs)
constexpr int F1_PREF = 4;    // chunks prefetched in registers
constexpr int F1_KMAX = 16;

template <typename C> struct F1Params {
    GridGeom<C> g;            // n2 = n
    const void *src;
    void *dst;
    int64_t jobs, cpj;        // jobs, output chunks per job
    int vec_ok;
    C w[7];                   // 2r+1 weights, offset -r..r
};

// One job: output chunks [c0, c1) advanced by K steps, reading chunks
// c0 - 1 .. c1 (each fused level's halo is at most one chunk).  COH: loads
// bypass L1 (data other SMs wrote during the same launch).
template <int DT, int R, int K, bool COH>
__device__ __forceinline__ void fused1d_job(const typename Traits<DT>::S *__restrict__ src,
                                            typename Traits<DT>::S *__restrict__ dst, int64_t n, bool periodic,
                                            typename Traits<DT>::C bval, const typename Traits<DT>::C *wr, int64_t c0,
                                            int64_t c1, bool vec_ok, int lane) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    constexpr int V = Traits<DT>::V;
    constexpr int CW = 32 * V;
    static_assert(K * R <= CW, "halo: one chunk each side");
    const int64_t a0 = c0 - 1;                       // first chunk read (left halo)
    const int nsteps = (int)(c1 - c0) + 1 + K;
    const bool edge = a0 < 0 || (c1 + 1) * CW > n;   // touches the grid's ends
    C ring[F1_PREF][V];
    auto load = [&](int64_t a, C *out) {
        const int64_t x0 = a * CW + (int64_t)lane * V;
        if (vec_ok && x0 >= 0 && x0 + V <= n) {
            ldvec<DT, COH>(src + x0, out);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int64_t x = x0 + v;
                if (x >= 0 && x < n) out[v] = to_c(ldx<COH>(src + x));
                else if (periodic) out[v] = to_c(ldx<COH>(src + wrap_idx(x, n)));
                else out[v] = bval;
            }
        }
    };
#pragma unroll
    for (int q = 0; q < F1_PREF; ++q) load(a0 + q, ring[q]);
    C hold[K][V], tail[K][R];
#pragma unroll
    for (int s = 0; s < K; ++s) {
#pragma unroll
        for (int v = 0; v < V; ++v) hold[s][v] = C(0);
#pragma unroll
        for (int q = 0; q < R; ++q) tail[s][q] = C(0);
    }
    const int nsp = round_up_c(nsteps, F1_PREF);
    for (int i0 = 0; i0 < nsp; i0 += F1_PREF) {
#pragma unroll
        for (int ph = 0; ph < F1_PREF; ++ph) {
            const int64_t a = a0 + i0 + ph;          // incoming level-0 chunk
            C inc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) inc[v] = ring[ph][v];
            load(a + F1_PREF, ring[ph]);
#pragma unroll
            for (int s = 0; s < K; ++s) {
                // level s+1 of chunk a-s-1 from tail[s], hold[s] and the head of inc
                C ext[V + 2 * R];
#pragma unroll
                for (int v = 0; v < V; ++v) ext[R + v] = hold[s][v];
                // the value q + 1 places left of the lane's first element sits
                // in the lane d = q / V + 1 places down, or for lanes l < d in
                // the previous chunk (vrl, index R + l V - 1 - q); the value
                // q + 1 places right of its last element in the lane d up, or
                // for lanes l >= 32 - d at the head of the incoming chunk
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int d = q / V + 1;
                    C left = __shfl_sync(0xffffffffu, hold[s][V - 1 - q % V], (lane - d) & 31);
#pragma unroll
                    for (int l = 0; l < (R + V - 1) / V; ++l)
                        if (l < d && lane == l) left = tail[s][R + l * V - 1 - q];
                    ext[R - 1 - q] = left;
                    const C dn = __shfl_sync(0xffffffffu, hold[s][q % V], (lane + d) & 31);
                    const C head = __shfl_sync(0xffffffffu, inc[q % V], (lane + d) & 31);
                    ext[R + V + q] = lane >= 32 - d ? head : dn;
                }
                C out[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    C acc = op_mul(wr[0], ext[v]);
#pragma unroll
                    for (int o = 1; o <= 2 * R; ++o) acc = op_fma(wr[o], ext[v + o], acc);
                    out[v] = acc;
                }
                if (edge && !periodic) {
                    const int64_t x0 = (a - s - 1) * CW + (int64_t)lane * V;
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (x0 + v < 0 || x0 + v >= n) out[v] = bval;
                }
                // advance level s: vrl <- last r values of VS, VS <- incoming
#pragma unroll
                for (int q = 0; q < R; ++q)
                    tail[s][q] = __shfl_sync(0xffffffffu, hold[s][(32 * V - R + q) % V], (32 * V - R + q) / V);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    hold[s][v] = inc[v];
                    inc[v] = out[v];
                }
            }
            const int64_t cx = a - K;                // chunk completed at level K
            if (cx >= c0 && cx < c1) {
                const int64_t x0 = cx * CW + (int64_t)lane * V;
                if (vec_ok && x0 + V <= n) {
                    stvec<DT>(dst + x0, inc);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (x0 + v < n) dst[x0 + v] = from_c<S>(inc[v]);
                }
            }
        }
    }
}

template <int DT, int R, int K>
__global__ void __launch_bounds__(F1_NW * 32) fused1d_kernel(const __grid_constant__ F1Params<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    constexpr int CW = 32 * Traits<DT>::V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C wr[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) wr[j] = p.w[j];
    const int64_t n = p.g.n2;
    const int64_t nchunks = (n + CW - 1) / CW;
    for (int64_t job = (int64_t)blockIdx.x * F1_NW + warp; job < p.jobs; job += (int64_t)gridDim.x * F1_NW) {
        const int64_t c0 = job * p.cpj;
        const int64_t c1 = c0 + p.cpj < nchunks ? c0 + p.cpj : nchunks;
        fused1d_job<DT, R, K, false>(static_cast<const S *>(p.src), static_cast<S *>(p.dst), n,
                                     p.g.bkind == STENCIL_PERIODIC, p.g.bval, wr, c0, c1, p.vec_ok != 0, lane);
    }
}

template <typename C> struct F1MpParams {
    GridGeom<C> g;          // n2 = n
    const void *src0;       // input of pass 0
    void *dst_even;         // output of the passes p with (passes - 1 - p) even (includes the last)
    void *dst_odd;
    int passes;
    int cpj, tiles;         // output chunks per tile, tiles
    int vec_ok;
    int *status;
    MpCtl *ctl;             // ticket, abort flag, exit count
    int *done;              // [tiles]: passes each tile has finished (all left at zero by the last warp)
    C w[7];
};

// All `passes` passes of K steps in one persistent launch (1D form of
// fused2d_mp_kernel): warps take (pass, tile) items pass-major; an item of
// pass p waits (acquire, bounded) until the tiles holding chunks c0 - 1 ..
// c1 of pass p - 1 -- every chunk its stored outputs depend on -- have
// published, then publishes its own completion with release semantics.
// A job also reads (prefetches) chunks beyond c1; those values feed only
// outputs it does not store.
template <int DT, int R, int K>
__global__ void __launch_bounds__(F1_NW * 32) fused1d_mp_kernel(const __grid_constant__ F1MpParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    constexpr int CW = 32 * Traits<DT>::V;
    const int lane = threadIdx.x & 31;
    MpCtl *ctl = p.ctl;
    int *done = p.done;
    C wr[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) wr[j] = p.w[j];
    const int n = (int)p.g.n2;
    const int nchunks = (n + CW - 1) / CW;
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    const unsigned long long items = (unsigned long long)p.tiles * (unsigned)p.passes;
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
        const int pass = (int)(t / (unsigned)p.tiles), j = (int)(t % (unsigned)p.tiles);
        const int c0 = j * p.cpj, c1 = c0 + p.cpj < nchunks ? c0 + p.cpj : nchunks;
        if (pass > 0) {
            // elements [(c0 - 1) CW, (c1 + 1) CW): tiles of cpj CW elements
            const TileSpan sp = tile_span((c0 - 1) * CW, (c1 + 1) * CW, n, p.cpj * CW, periodic);
            bool ok = true;
            for (int e = lane; e < sp.count(); e += 32) ok = ok && wait_counter(&done[sp.at(e)], pass, &ctl->abort);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) {
                    atomicExch(&ctl->abort, 1);
                    record_status(p.status, kStatusTimeout);
                }
                break;
            }
            __syncwarp();   // every lane's acquire precedes every lane's (L2) reads
        }
        const bool from_even = ((p.passes - pass) & 1) == 0;   // pass - 1 wrote dst_even
        const S *src = static_cast<const S *>(pass == 0 ? p.src0 : from_even ? p.dst_even : p.dst_odd);
        S *dst = static_cast<S *>(((p.passes - 1 - pass) & 1) == 0 ? p.dst_even : p.dst_odd);
        fused1d_job<DT, R, K, true>(src, dst, n, periodic, p.g.bval, wr, c0, c1, p.vec_ok != 0, lane);
        __syncwarp();
        if (lane == 0) red_release_add(&done[j], 1);
    }
    // the last warp out leaves the counters at zero for the next launch
    __syncwarp();
    int last = 0;
    if (lane == 0) last = worker_exit_is_last(&ctl->exited, gridDim.x * F1_NW);
    if (__shfl_sync(0xffffffffu, last, 0)) {
        for (int i = lane; i < p.tiles; i += 32) done[i] = 0;
        if (lane == 0) {
            ctl->ticket = 0ull;
            ctl->abort = 0;
            ctl->exited = 0u;
        }
    }
}

template <int DT, int R, int K>
static cudaError_t launch_f1_t(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    using C = typename Traits<DT>::C;
    constexpr int CW = 32 * Traits<DT>::V;
    F1Params<C> p;
    p.g.n0 = 1;
    p.g.n1 = 1;
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.src = src;
    p.dst = dst;
    p.vec_ok = ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
    if (P.np > (int)(sizeof(p.w) / sizeof(p.w[0]))) return cudaErrorInvalidValue;   // weights fit the parameter block
    for (int j = 0; j < 2 * R + 1; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    const int64_t nchunks = (P.n[2] + CW - 1) / CW;
    // about four jobs per warp slot, each at least 4 (K + 1) chunks long
    const int64_t slots = (int64_t)P.sm_count * 16 * F1_NW;
    int64_t cpj = (nchunks + 4 * slots - 1) / (4 * slots);
    if (cpj < 4 * (K + 1)) cpj = 4 * (K + 1);
    p.cpj = cpj;
    p.jobs = (nchunks + cpj - 1) / cpj;
    int64_t grid = (p.jobs + F1_NW - 1) / F1_NW;
    if (grid > (int64_t)P.sm_count * 16) grid = (int64_t)P.sm_count * 16;
    fused1d_kernel<DT, R, K><<<(unsigned)grid, F1_NW * 32, 0, st>>>(p);
    return cudaGetLastError();
}

// Chunks per tile of the persistent form: about three tiles per resident
// warp, and at least 2k (a job streams k + 1 chunks beyond its outputs).
template <int DT, int R, int K>
static cudaError_t launch_f1mp_t(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int passes,
                                 cudaStream_t st) {
    using C = typename Traits<DT>::C;
    constexpr int CW = 32 * Traits<DT>::V;
    if (!fused1d_multi_ok(P, K) || passes < 1) return cudaErrorNotSupported;
    F1MpParams<C> p;
    p.g.n0 = 1;
    p.g.n1 = 1;
    p.g.n2 = P.n[2];
    p.g.bkind = P.bkind;
    p.g.bval = conv_w<C>(P.bval);
    p.src0 = src0;
    p.dst_even = dst_even;
    p.dst_odd = dst_odd;
    p.passes = passes;
    p.status = P.d_status;
    if (P.np > (int)(sizeof(p.w) / sizeof(p.w[0]))) return cudaErrorInvalidValue;   // weights fit the parameter block
    for (int j = 0; j < 2 * R + 1; ++j) p.w[j] = conv_w<C>(P.w_eval[j]);
    p.vec_ok = ((uintptr_t)src0 % 16 == 0) && ((uintptr_t)dst_even % 16 == 0) && ((uintptr_t)dst_odd % 16 == 0);
    const int64_t nchunks = (P.n[2] + CW - 1) / CW;
    const int64_t slots = (int64_t)P.sm_count * 16 * F1_NW;
    int64_t cpj = P.tile_rows > 0 ? P.tile_rows : std::max<int64_t>((nchunks + 3 * slots - 1) / (3 * slots), 2 * K);
    if (cpj > nchunks) cpj = nchunks;
    p.cpj = (int)cpj;
    p.tiles = (int)((nchunks + cpj - 1) / cpj);
    cudaError_t e = ensure_mp_state(P, p.tiles, st);
    if (e != cudaSuccess) return e;
    p.ctl = static_cast<MpCtl *>(P.d_mp);
    p.done = reinterpret_cast<int *>(static_cast<char *>(P.d_mp) + sizeof(MpCtl));
    // warps for about two passes of tiles: more would take tickets many
    // passes ahead and only poll their dependencies
    const int64_t jobs = std::min<int64_t>((int64_t)p.tiles * passes, 2 * (int64_t)p.tiles);
    int64_t grid = (jobs + F1_NW - 1) / F1_NW;
    if (grid > (int64_t)P.sm_count * 16) grid = (int64_t)P.sm_count * 16;
    fused1d_mp_kernel<DT, R, K><<<(unsigned)grid, F1_NW * 32, 0, st>>>(p);
    return cudaGetLastError();
}

// Largest fusion depth built: 16, or 8 for the half-precision storage types.
template <int DT> constexpr int f1_kmax() { return (DT == STENCIL_BF16 || DT == STENCIL_F16) ? 8 : F1_KMAX; }

// Fusion depths K..f1_kmax of one radius (compile-time recursion over K).
template <int DT, int R, int K>
cudaError_t launch_f1_kr(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    if constexpr (K > f1_kmax<DT>()) {
        return cudaErrorInvalidValue;
    } else {
        if (k == K) return launch_f1_t<DT, R, K>(P, src, dst, st);
        return launch_f1_kr<DT, R, K + 1>(P, src, dst, k, st);
    }
}

template <int DT, int R, int K>
cudaError_t launch_f1mp_kr(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                           cudaStream_t st) {
    if constexpr (K > f1_kmax<DT>()) {
        return cudaErrorInvalidValue;
    } else {
        if (k == K) return launch_f1mp_t<DT, R, K>(P, src0, de, dof, passes, st);
        return launch_f1mp_kr<DT, R, K + 1>(P, src0, de, dof, k, passes, st);
    }
}

template <int DT>
cudaError_t launch_f1_dt(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (P.r) {
        case 1: return launch_f1_kr<DT, 1, 1>(P, src, dst, k, st);
        case 2: return launch_f1_kr<DT, 2, 1>(P, src, dst, k, st);
        case 3: return launch_f1_kr<DT, 3, 1>(P, src, dst, k, st);
    }
    return cudaErrorInvalidValue;
}

template <int DT>
cudaError_t launch_f1mp_dt(const stencil_plan_s &P, const void *src0, void *de, void *dof, int k, int passes,
                           cudaStream_t st) {
    switch (P.r) {
        case 1: return launch_f1mp_kr<DT, 1, 1>(P, src0, de, dof, k, passes, st);
        case 2: return launch_f1mp_kr<DT, 2, 1>(P, src0, de, dof, k, passes, st);
        case 3: return launch_f1mp_kr<DT, 3, 1>(P, src0, de, dof, k, passes, st);
    }
    return cudaErrorInvalidValue;
}

// one translation unit per storage type (k_fused1d_<dtype>.cu)
#define SG_DECL_F1(DT)                                                                             \
    cudaError_t launch_f1_##DT(const stencil_plan_s &, const void *, void *, int, cudaStream_t);  \
    cudaError_t launch_f1mp_##DT(const stencil_plan_s &, const void *, void *, void *, int, int, cudaStream_t);
SG_DECL_F1(F32)
SG_DECL_F1(F64)
SG_DECL_F1(BF16)
SG_DECL_F1(F16)
SG_DECL_F1(I32)
#undef SG_DECL_F1

}  // namespace sg
