// k_fused1d.cu -- 1D Jacobi sweep with K time steps fused per pass.
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
#include <string>

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

constexpr int F1_NW = 4;      // warps per CTA (independent jobs)
constexpr int F1_PREF = 4;    // chunks prefetched in registers
constexpr int F1_KMAX = 8;

template <typename C> struct F1Params {
    GridGeom<C> g;            // n2 = n
    const void *src;
    void *dst;
    int64_t jobs, cpj;        // jobs, output chunks per job
    int vec_ok;
    C w[7];                   // 2r+1 weights, offset -r..r
};

template <int DT, int R, int K>
__global__ void __launch_bounds__(F1_NW * 32) fused1d_kernel(const __grid_constant__ F1Params<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    constexpr int V = Traits<DT>::V;
    constexpr int CW = 32 * V;
    static_assert(K * R <= CW && R <= V, "halo");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const S *__restrict__ src = static_cast<const S *>(p.src);
    S *__restrict__ dst = static_cast<S *>(p.dst);
    const int64_t n = p.g.n2;
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    const C bval = p.g.bval;
    const bool vec_ok = p.vec_ok != 0;
    C wr[2 * R + 1];
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) wr[j] = p.w[j];
    const int64_t nchunks = (n + CW - 1) / CW;

    for (int64_t job = (int64_t)blockIdx.x * F1_NW + warp; job < p.jobs; job += (int64_t)gridDim.x * F1_NW) {
        const int64_t c0 = job * p.cpj;
        const int64_t c1 = c0 + p.cpj < nchunks ? c0 + p.cpj : nchunks;
        const int64_t a0 = c0 - 1;                       // first chunk read (left halo)
        const int nsteps = (int)(c1 - c0) + 1 + K;
        const bool edge = a0 < 0 || (c1 + 1) * CW > n;   // touches the grid's ends
        C ring[F1_PREF][V];
        auto load = [&](int64_t a, C *out) {
            const int64_t x0 = a * CW + (int64_t)lane * V;
            if (vec_ok && x0 >= 0 && x0 + V <= n) {
                ldvec<DT, false>(src + x0, out);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int64_t x = x0 + v;
                    if (x >= 0 && x < n) out[v] = to_c(__ldg(src + x));
                    else if (periodic) out[v] = to_c(__ldg(src + wrap_idx(x, n)));
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
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const C up = __shfl_up_sync(0xffffffffu, hold[s][V - 1 - q], 1);
                        ext[R - 1 - q] = lane == 0 ? tail[s][R - 1 - q] : up;
                        const C dn = __shfl_down_sync(0xffffffffu, hold[s][q], 1);
                        const C head = __shfl_sync(0xffffffffu, inc[q], 0);
                        ext[R + V + q] = lane == 31 ? head : dn;
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
                    for (int q = 0; q < R; ++q) tail[s][q] = __shfl_sync(0xffffffffu, hold[s][V - R + q], 31);
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

template <int DT, int R>
static cudaError_t launch_f1_k(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (k) {
        case 1: return launch_f1_t<DT, R, 1>(P, src, dst, st);
        case 2: return launch_f1_t<DT, R, 2>(P, src, dst, st);
        case 3: return launch_f1_t<DT, R, 3>(P, src, dst, st);
        case 4: return launch_f1_t<DT, R, 4>(P, src, dst, st);
        case 5: return launch_f1_t<DT, R, 5>(P, src, dst, st);
        case 6: return launch_f1_t<DT, R, 6>(P, src, dst, st);
        case 7: return launch_f1_t<DT, R, 7>(P, src, dst, st);
        case 8: return launch_f1_t<DT, R, 8>(P, src, dst, st);
    }
    return cudaErrorInvalidValue;
}

template <int DT>
static cudaError_t launch_f1_dt(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (P.r) {
        case 1: return launch_f1_k<DT, 1>(P, src, dst, k, st);
        case 2: return launch_f1_k<DT, 2>(P, src, dst, k, st);
    }
    return cudaErrorInvalidValue;
}

int fused1d_max_k(const stencil_plan_s &P) {
    if (P.dim != 1 || P.r > 2) return 0;
    return F1_KMAX;
}

cudaError_t launch_fused1d(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F64: return launch_f1_dt<STENCIL_F64>(P, src, dst, k, st);
        case STENCIL_F32: return launch_f1_dt<STENCIL_F32>(P, src, dst, k, st);
        case STENCIL_BF16: return launch_f1_dt<STENCIL_BF16>(P, src, dst, k, st);
        case STENCIL_F16: return launch_f1_dt<STENCIL_F16>(P, src, dst, k, st);
        case STENCIL_I32: return launch_f1_dt<STENCIL_I32>(P, src, dst, k, st);
    }
    return cudaErrorInvalidValue;
}

std::string fused1d_describe(const stencil_plan_s &P, int k) {
    return "fused1d(warp-streamed vector sets, k=" + std::to_string(k) + ")";
}

}  // namespace sg
