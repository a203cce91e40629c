// k_adjoint.cu -- reverse-mode derivative of the T-step sweep (FP32 plans).
//
// Not in the paper.  The sweep is u_{t+1} = A u_t + c (c: the Dirichlet
// boundary's constant contribution).  For a loss L(u_T) with lam_T = dL/du_T:
//     dL/dw_j += sum_x lam_{t+1}[x] * u_t(x + o_j)      (boundary values included)
//     lam_t    = A^T lam_{t+1},  (A^T lam)[y] = sum_j w_j lam[y - o_j]
// for t = T-1 .. 0, and dL/du_0 = lam_0.  A^T is the stencil with reflected
// offsets; lam outside a Dirichlet domain is 0 (boundary cells are constants),
// periodic indices wrap.  One kernel does both lines of a backward step: it
// reads lam_{t+1} and u_t once, writes lam_t, and adds its weight-gradient
// terms (FP32 per thread over its four points, widened to FP64 for the block
// sums) into per-block FP64 partials that persist across the steps; a final
// one-block kernel sums the partials in a fixed order.
//
// Forward states come from checkpoints taken while the forward sweep runs
// (stencil_run_checkpointed: the fused sweep in segments of c steps, each
// segment's result kept): the backward sweep walks the segments last to
// first, recomputes a segment's c - 1 inner states from its checkpoint one
// step per launch, then runs its c transposed steps.  stencil_adjoint_run
// takes the checkpoints itself first.
#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "k_adjoint3d.cuh"
#include "plan.h"

namespace sg {

constexpr int ADJ_THREADS = 256;
constexpr int ADJ_VX = 4;

struct AdjParams {
    const float *lam_in;   // lam_{t+1}
    const float *u;        // u_t
    float *lam_out;        // lam_t
    double *partials;      // [blocks][np]
    int64_t n0, n1, n2;
    int bkind;
    float bval;
    int first;             // 1: overwrite partials, 0: add
    int vec_ok;            // rows and the three pointers allow float4 access
    float w[kMaxPts];      // evaluation (lexicographic) order
};

// Launch shape of one backward step: the rows kernel (grid-stride over
// (plane, row block) pairs) where the extents allow it, else the generic one.
struct AdjShape {
    bool rows;
    bool z3;               // the z-streamed 3D kernel (k_adjoint3d.cuh)
    dim3 grid, block;
    int nblocks;           // blocks = partial-sum slots
};

template <int D, int R, int PAT>
__global__ void __launch_bounds__(ADJ_THREADS) adjoint_step_kernel(const __grid_constant__ AdjParams p) {
    using Sh = Shape<D, R, PAT>;
    constexpr int NP = Sh::npts;
    constexpr int NZ = D == 3 ? 2 * R + 1 : 1, NY = D >= 2 ? 2 * R + 1 : 1, SP = ADJ_VX + 2 * R;
    __shared__ double red[ADJ_THREADS / 32][NP];
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2;
    const bool periodic = p.bkind == STENCIL_PERIODIC;
    const int64_t groups = (n2 + ADJ_VX - 1) / ADJ_VX;
    const int64_t rows = n0 * n1;
    const int64_t items = rows * groups;
    float gw[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) gw[j] = 0.f;
    for (int64_t it = blockIdx.x * (int64_t)ADJ_THREADS + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * ADJ_THREADS) {
        const int64_t g = it % groups, row = it / groups;
        const int64_t i1 = row % n1, i0 = row / n1;
        const int64_t x0 = g * ADJ_VX;
        float lam[NZ][NY][SP], uu[NZ][NY][SP];
#pragma unroll
        for (int jz = 0; jz < NZ; ++jz)
#pragma unroll
            for (int jy = 0; jy < NY; ++jy) {
                const int oz = D == 3 ? jz - R : 0, oy = D >= 2 ? jy - R : 0;
                if (!Sh::inc(oz, oy, 0)) continue;
                const bool halo = PAT == STENCIL_BOX || (oz == 0 && oy == 0);
                int64_t z = i0 + oz, y = i1 + oy;
                bool ok = true;
                if (z < 0 || z >= n0) { if (periodic) z = wrap_idx(z, n0); else ok = false; }
                if (y < 0 || y >= n1) { if (periodic) y = wrap_idx(y, n1); else ok = false; }
                const int64_t base = (z * n1 + y) * n2;
#pragma unroll
                for (int q = 0; q < SP; ++q) {
                    if (!halo && (q < R || q >= R + ADJ_VX)) continue;
                    int64_t x = x0 - R + q;
                    bool okx = ok;
                    if (x < 0 || x >= n2) { if (periodic) x = wrap_idx(x, n2); else okx = false; }
                    lam[jz][jy][q] = okx ? __ldg(p.lam_in + base + x) : 0.f;
                    uu[jz][jy][q] = okx ? __ldg(p.u + base + x) : p.bval;
                }
            }
        // lam_t[x] = sum_o w_o lam_{t+1}[x - o]; gw_o += lam_{t+1}[x] * u_t(x + o)
        float acc[ADJ_VX];
        bool first = true;
#pragma unroll
        for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz)
#pragma unroll
            for (int oy = (D >= 2 ? -R : 0); oy <= (D >= 2 ? R : 0); ++oy)
#pragma unroll
                for (int ox = -R; ox <= R; ++ox) {
                    if (!Sh::inc(oz, oy, ox)) continue;
                    const int j = Sh::widx(oz, oy, ox);
                    const float w = p.w[j];
                    const int rz = D == 3 ? R - oz : 0, ry = D >= 2 ? R - oy : 0;   // row of x - o
                    const int fz = D == 3 ? R + oz : 0, fy = D >= 2 ? R + oy : 0;   // row of x + o
#pragma unroll
                    for (int v = 0; v < ADJ_VX; ++v) {
                        const float l = lam[rz][ry][R + v - ox];
                        acc[v] = first ? __fmul_rn(w, l) : __fmaf_rn(w, l, acc[v]);
                        if (x0 + v < n2) gw[j] = __fmaf_rn(lam[D == 3 ? R : 0][D >= 2 ? R : 0][R + v], uu[fz][fy][R + v + ox], gw[j]);
                    }
                    first = false;
                }
        float *out = p.lam_out + (i0 * n1 + i1) * n2;
#pragma unroll
        for (int v = 0; v < ADJ_VX; ++v)
            if (x0 + v < n2) out[x0 + v] = acc[v];
    }
    // block sums of the weight-gradient terms: each thread's FP32 sum over
    // its own points of this step, then FP64 from the warp tree up
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        double v = (double)gw[j];
        for (int o = 16; o > 0; o >>= 1) v = v + __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double s = 0.0;
        for (int wi = 0; wi < ADJ_THREADS / 32; ++wi) s += red[wi][threadIdx.x];
        double *dst = p.partials + (size_t)blockIdx.x * NP + threadIdx.x;
        *dst = p.first ? s : *dst + s;
    }
}

// The same backward step for grids with moderate extents (each extent
// > 2r + RB + 2, 32-bit indices): a block of TX x TY threads covers TX groups
// of 4 x-points and TY x RB rows; blocks walk the (plane, row block) pairs
// with a grid stride, so the number of blocks -- and of FP64 partials -- stays
// a few per SM.  Plane and row indices are uniform across a warp; halo rows
// and columns wrap by one extent (periodic) or read 0 / the boundary value.
// resident blocks per SM the register allocation must allow (r = 2 and the
// 3D box keep larger neighbourhoods in registers)
constexpr int adj_min_blocks(int d, int r, int pat) { return r == 1 && !(d == 3 && pat == STENCIL_BOX) ? 3 : 1; }

template <int D, int R, int PAT, int RB>
__global__ void __launch_bounds__(ADJ_THREADS, adj_min_blocks(D, R, PAT)) adjoint_rows_kernel(const __grid_constant__ AdjParams p) {
    using Sh = Shape<D, R, PAT>;
    constexpr int NP = Sh::npts, VX = ADJ_VX;
    constexpr int NZ = D == 3 ? 2 * R + 1 : 1;
    constexpr int NY = D >= 2 ? RB + 2 * R : 1;
    constexpr int SP = VX + 2 * R;
    __shared__ double red[ADJ_THREADS / 32][NP];
    const int n0 = (int)p.n0, n1 = (int)p.n1, n2 = (int)p.n2;
    const bool periodic = p.bkind == STENCIL_PERIODIC;
    const float bval = p.bval;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int rows = (n1 + RB * (int)blockDim.y - 1) / (RB * (int)blockDim.y);   // row blocks per plane
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
    const bool full = x0 + VX <= n2;
    const bool vec = full && p.vec_ok;
    float gw[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) gw[j] = 0.f;
    for (int rbk = blockIdx.y; rbk < n0 * rows; rbk += gridDim.y) {
        const int i0 = rbk / rows;
        const int i1b = ((rbk - i0 * rows) * (int)blockDim.y + (int)threadIdx.y) * RB;
        if (x0 >= n2 || i1b >= n1) continue;
        float lam[NZ][NY][SP], uu[NZ][NY][SP];
#pragma unroll
        for (int jz = 0; jz < NZ; ++jz) {
            const int oz = D == 3 ? jz - R : 0;
#pragma unroll
            for (int jy = 0; jy < NY; ++jy) {
                bool used = false, halo = false;
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    const int oy = D >= 2 ? jy - R - b : 0;
                    if (D >= 2 && (oy < -R || oy > R)) continue;
                    if (Sh::inc(oz, oy, 0)) used = true;
                    if (PAT == STENCIL_BOX || (oz == 0 && oy == 0)) halo = true;
                }
                if (!used) continue;
                int z = i0 + oz, y = D >= 2 ? i1b - R + jy : 0;
                bool ok = true;
                if (z < 0) { z += n0; ok = periodic; }
                else if (z >= n0) { z -= n0; ok = periodic; }
                if (y < 0) { y += n1; ok = ok && periodic; }
                else if (y >= n1) { y -= n1; ok = ok && periodic; }
                float *lr = lam[jz][jy], *ur = uu[jz][jy];
                if (!ok) {
#pragma unroll
                    for (int q = 0; q < SP; ++q) { lr[q] = 0.f; ur[q] = bval; }
                    continue;
                }
                const size_t base = ((size_t)z * n1 + y) * n2;
                const float *lp = p.lam_in + base, *up = p.u + base;
                if (vec) {
                    const float4 a = __ldg(reinterpret_cast<const float4 *>(lp + x0));
                    const float4 c = __ldg(reinterpret_cast<const float4 *>(up + x0));
                    lr[R] = a.x; lr[R + 1] = a.y; lr[R + 2] = a.z; lr[R + 3] = a.w;
                    ur[R] = c.x; ur[R + 1] = c.y; ur[R + 2] = c.z; ur[R + 3] = c.w;
                } else {
#pragma unroll
                    for (int q = 0; q < VX; ++q) {   // last, partial group: wrap or outside value
                        const int x = x0 + q;
                        const bool in = x < n2;
                        const int xx = in ? x : x - n2;
                        lr[R + q] = (in || periodic) ? __ldg(lp + xx) : 0.f;
                        ur[R + q] = (in || periodic) ? __ldg(up + xx) : bval;
                    }
                }
                if (halo) {
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        int xl = x0 - R + q, xr = x0 + VX + q;
                        const bool il = xl >= 0, ir = xr < n2;
                        xl = il ? xl : xl + n2;
                        xr = ir ? xr : xr - n2;
                        lr[q] = (il || periodic) ? __ldg(lp + xl) : 0.f;
                        ur[q] = (il || periodic) ? __ldg(up + xl) : bval;
                        lr[R + VX + q] = (ir || periodic) ? __ldg(lp + xr) : 0.f;
                        ur[R + VX + q] = (ir || periodic) ? __ldg(up + xr) : bval;
                    }
                }
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int yo = D >= 2 ? i1b + b : 0;
            if (yo >= n1) break;
            const int cz = D == 3 ? R : 0, cy = D >= 2 ? R + b : 0;   // this output's own row
            float acc[VX];
            bool first = true;
#pragma unroll
            for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz)
#pragma unroll
                for (int oy = (D >= 2 ? -R : 0); oy <= (D >= 2 ? R : 0); ++oy)
#pragma unroll
                    for (int ox = -R; ox <= R; ++ox) {
                        if (!Sh::inc(oz, oy, ox)) continue;
                        const int j = Sh::widx(oz, oy, ox);
                        const float w = p.w[j];
                        const float *lrow = lam[D == 3 ? R - oz : 0][D >= 2 ? R + b - oy : 0];   // row of x - o
                        const float *urow = uu[D == 3 ? R + oz : 0][D >= 2 ? R + b + oy : 0];    // row of x + o
#pragma unroll
                        for (int v = 0; v < VX; ++v) {
                            const float l = lrow[R + v - ox];
                            acc[v] = first ? __fmul_rn(w, l) : __fmaf_rn(w, l, acc[v]);
                            if (full || x0 + v < n2) gw[j] = __fmaf_rn(lam[cz][cy][R + v], urow[R + v + ox], gw[j]);
                        }
                        first = false;
                    }
            float *out = p.lam_out + ((size_t)i0 * n1 + yo) * n2;
            if (vec) {
                *reinterpret_cast<float4 *>(out + x0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
            } else {
#pragma unroll
                for (int v = 0; v < VX; ++v)
                    if (x0 + v < n2) out[x0 + v] = acc[v];
            }
        }
    }
    // block sums of the weight-gradient terms, fixed order: each thread's
    // FP32 sum over its own points of this step (a few dozen products: FP64
    // per product would keep the FP64 pipe -- 2 operations per clock per SM
    // on this GPU -- busy for longer than the whole step), then FP64 from the
    // warp tree up, across warps, blocks and steps
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        double v = (double)gw[j];
        for (int o = 16; o > 0; o >>= 1) v = v + __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (tid < NP) {
        double s = 0.0;
        for (int wi = 0; wi < ADJ_THREADS / 32; ++wi) s += red[wi][tid];
        double *dst = p.partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * NP + tid;
        *dst = p.first ? s : *dst + s;
    }
}

// grad_w[compact j] = sum over blocks of partials[b][eval j], fixed order
__global__ void adjoint_wgrad_final(const double *__restrict__ partials, int nblocks, int np,
                                    const int *__restrict__ eval_to_compact, double *grad_w) {
    __shared__ double sh[256];
    for (int j = 0; j < np; ++j) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 256) s += partials[(size_t)b * np + j];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) grad_w[eval_to_compact[j]] = sh[0];
        __syncthreads();
    }
}

// rows per thread in the rows kernel: two where the loaded rows stay few
constexpr int adj_rb(int d, int pat) { return d == 2 ? 2 : 1; }

static AdjShape adj_shape(const stencil_plan_s &P) {
    AdjShape a;
    a.z3 = false;
    // 3D stencils of up to 27 points: the z-streamed kernel, two CTAs per SM
    // at radius 1 (96 KB of planes each), one at radius 2 (149 KB)
    if (P.dim == 3 && P.np <= 27 && P.n[0] < (1ll << 30) && P.n[1] < (1ll << 30) && P.n[2] < (1ll << 30) &&
        (P.n[2] + A3_TX - 1) / A3_TX * ((P.n[1] + A3_TY - 1) / A3_TY) < (1ll << 30)) {
        a.z3 = true;
        a.rows = false;
        a.nblocks = P.sm_count * (P.r == 1 ? 2 : 1);
        a.grid = dim3((unsigned)a.nblocks, 1, 1);
        a.block = dim3(A3_THREADS, 1, 1);
        return a;
    }
    const int64_t n0 = P.n[0], n1 = P.n[1], n2 = P.n[2], r = P.r;
    const int rb = adj_rb(P.dim, P.pattern);
    const int64_t groups = (n2 + ADJ_VX - 1) / ADJ_VX;
    const int tx = (int)std::min<int64_t>(ADJ_THREADS, (groups + 31) / 32 * 32);
    const int ty = ADJ_THREADS / tx;
    const int64_t bx = (groups + tx - 1) / tx;
    const int64_t rowblocks = n0 * ((n1 + (int64_t)rb * ty - 1) / ((int64_t)rb * ty));
    a.rows = (P.dim < 3 || n0 > 2 * r + 2) && (P.dim < 2 || n1 > 2 * r + rb + 2) && n2 >= 2 * (ADJ_VX + r) &&
             n0 < (1ll << 30) && n1 < (1ll << 30) && n2 < (1ll << 30) && rowblocks < (1ll << 31) && bx <= 65535;
    if (a.rows) {
        // about 16 blocks per SM in all, each walking several row blocks
        const int64_t want = std::max<int64_t>(1, (int64_t)P.sm_count * 16 / bx);
        const int64_t by = std::min<int64_t>(std::min<int64_t>(rowblocks, want), 65535);
        a.grid = dim3((unsigned)bx, (unsigned)by, 1);
        a.block = dim3((unsigned)tx, (unsigned)ty, 1);
        a.nblocks = (int)(bx * by);
    } else {
        const int64_t items = n0 * n1 * groups;
        int64_t nb = (items + ADJ_THREADS - 1) / ADJ_THREADS;
        nb = std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)P.sm_count * 8));
        a.grid = dim3((unsigned)nb, 1, 1);
        a.block = dim3(ADJ_THREADS, 1, 1);
        a.nblocks = (int)nb;
    }
    return a;
}

template <int D, int R, int PAT>
static cudaError_t launch_adj_t(const AdjParams &p, const AdjShape &a, cudaStream_t st) {
    if (a.rows) adjoint_rows_kernel<D, R, PAT, adj_rb(D, PAT)><<<a.grid, a.block, 0, st>>>(p);
    else adjoint_step_kernel<D, R, PAT><<<a.grid, a.block, 0, st>>>(p);
    return cudaGetLastError();
}

template <int R, int PAT>
static cudaError_t launch_adj3_t(const Adj3Params &q, const AdjShape &a, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(adjoint3d_kernel<R, PAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             A3Geo<R>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    adjoint3d_kernel<R, PAT><<<a.grid, a.block, A3Geo<R>::SMEM, st>>>(q);
    return cudaGetLastError();
}

static cudaError_t launch_adj(const stencil_plan_s &P, const AdjParams &p, const AdjShape &a, cudaStream_t st) {
    if (a.z3) {
        Adj3Params q;
        q.lam_in = p.lam_in;
        q.u = p.u;
        q.lam_out = p.lam_out;
        q.partials = p.partials;
        q.nx = (int)P.n[2];
        q.ny = (int)P.n[1];
        q.nz = (int)P.n[0];
        q.tiles_x = (int)((P.n[2] + A3_TX - 1) / A3_TX);
        q.tiles_y = (int)((P.n[1] + A3_TY - 1) / A3_TY);
        q.periodic = P.bkind == STENCIL_PERIODIC;
        q.bval = p.bval;
        q.first = p.first;
        q.vec = p.vec_ok;
        for (int j = 0; j < P.np; ++j) q.w[j] = p.w[j];
        if (P.r == 1) return P.pattern == STENCIL_BOX ? launch_adj3_t<1, STENCIL_BOX>(q, a, st)
                                                      : launch_adj3_t<1, STENCIL_STAR>(q, a, st);
        if (P.r == 2 && P.pattern == STENCIL_STAR) return launch_adj3_t<2, STENCIL_STAR>(q, a, st);
        return cudaErrorInvalidValue;
    }
    const bool box = P.pattern == STENCIL_BOX;
#define SG_ADJ(DD, RR)                                                                                  \
    if (P.dim == DD && P.r == RR) return box ? launch_adj_t<DD, RR, STENCIL_BOX>(p, a, st)              \
                                             : launch_adj_t<DD, RR, STENCIL_STAR>(p, a, st);
    SG_ADJ(1, 1) SG_ADJ(1, 2) SG_ADJ(2, 1) SG_ADJ(2, 2) SG_ADJ(3, 1) SG_ADJ(3, 2)
#undef SG_ADJ
    return cudaErrorInvalidValue;
}

}  // namespace sg

using namespace sg;

namespace sg {

static stencil_status_t adj_check(const stencil_plan_s *P, int64_t T, int32_t c) {
    if (P->dtype != STENCIL_F32 || P->r > 2) {
        set_error("the adjoint supports F32 plans of radius 1 or 2");
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (T > 0 && (c < 1 || c > T)) {
        set_error("ckpt_every must be in 1..T");
        return STENCIL_ERR_INVALID_ARG;
    }
    return STENCIL_OK;
}

// the forward sweep in segments of c steps, segment m's result stored as
// checkpoint m (m < M - 1) or u_T (the last)
static stencil_status_t forward_ckpt(stencil_plan_s *P, const void *u0, void *uT, int64_t T, int c, void *ckpts,
                                     void *stream) {
    const size_t gb = P->grid_bytes;
    const int64_t M = (T + c - 1) / c;
    const void *src = u0;
    for (int64_t m = 0; m < M; ++m) {
        void *dst = m == M - 1 ? uT : static_cast<void *>(static_cast<char *>(ckpts) + (size_t)m * gb);
        const int64_t steps = std::min<int64_t>(c, T - m * c);
        stencil_status_t s = stencil_run(P, src, dst, steps, stream);
        if (s != STENCIL_OK) return s;
        src = dst;
    }
    return STENCIL_OK;
}

// The backward sweep from checkpoints (u0 = checkpoint 0, ckpts[m - 1] =
// the state after m c steps): each segment, last to first, recomputes its
// c - 1 inner states one step per launch (the plan's fused kernels at k = 1)
// and then runs its c transposed steps.
static stencil_status_t backward_from_ckpts(stencil_plan_s *P, const void *u0, const void *ckpts,
                                            const void *grad_uT, int64_t T, int c, void *grad_u0, double *grad_w,
                                            void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t gb = P->grid_bytes;
    if (T == 0) {
        cudaError_t e = cudaMemcpyAsync(grad_u0, grad_uT, gb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(grad_w, 0, sizeof(double) * P->np, st);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
        return STENCIL_OK;
    }
    const int64_t M = (T + c - 1) / c;
    // workspace: c - 1 recomputed states, two lam grids, the partials
    const size_t ngrids = (size_t)(c - 1) + 2;
    const AdjShape shape = adj_shape(*P);
    const int nblocks = shape.nblocks;
    const size_t need = ngrids * gb + 256 + sizeof(double) * (size_t)nblocks * P->np + sizeof(int) * P->np;
    if (P->adj_ws_bytes < need) {
        cudaFree(P->adj_ws);
        P->adj_ws = nullptr;
        P->adj_ws_bytes = 0;
        if (cudaMalloc(&P->adj_ws, need) != cudaSuccess) {
            cudaGetLastError();
            set_error("adjoint workspace allocation of " + std::to_string(need) + " bytes failed");
            return STENCIL_ERR_OOM;
        }
        P->adj_ws_bytes = need;
    }
    char *ws = static_cast<char *>(P->adj_ws);
    auto grid_at = [&](size_t i) { return static_cast<void *>(ws + i * gb); };
    double *partials = reinterpret_cast<double *>(ws + ((ngrids * gb + 255) / 256) * 256);
    int *e2c = reinterpret_cast<int *>(partials + (size_t)nblocks * P->np);
    std::vector<int> h_e2c(P->eval_to_compact, P->eval_to_compact + P->np);
    cudaError_t e = cudaMemcpyAsync(e2c, h_e2c.data(), sizeof(int) * P->np, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
    auto ckpt = [&](int64_t m) -> const void * {
        return m == 0 ? u0 : static_cast<const void *>(static_cast<const char *>(ckpts) + (size_t)(m - 1) * gb);
    };
    auto seg = [&](int i) -> void * { return grid_at((size_t)(i - 1)); };   // i = 1..c-1
    void *lam[2] = {grid_at((size_t)(c - 1)), grid_at((size_t)c)};
    AdjParams p;
    p.n0 = P->n[0];
    p.n1 = P->n[1];
    p.n2 = P->n[2];
    p.bkind = P->bkind;
    p.bval = (float)P->bval;
    p.partials = partials;
    for (int j = 0; j < P->np; ++j) p.w[j] = (float)P->w_eval[j];
    // fused recompute where the plan's fused 3D kernel exists for this
    // geometry and the tuner (if it ran) did not find the plain sweep faster
    const bool all_levels = P->dim == 3 && P->r == 1 && fused3d_max_k(*P) >= 1 && !P->tuned_plain;
    if (all_levels) {
        stencil_status_t s = ensure_status_word(P);
        if (s != STENCIL_OK) return s;
    }
    const float *lam_next = static_cast<const float *>(grad_uT);
    int li = 0;
    bool first = true;
    for (int64_t m = M - 1; m >= 0; --m) {
        const int64_t t0 = m * c, t1 = std::min<int64_t>(T, t0 + c);
        // the segment's inner states t0 + 1 .. t1 - 1: 3D radius-1 plans run
        // fused passes of up to 4 steps that store every level; otherwise one
        // step per launch
        int64_t t = t0;
        const void *src = ckpt(m);
        while (t + 1 < t1) {
            const int kk = (int)std::min<int64_t>(4, t1 - 1 - t);
            void *lv[4] = {nullptr, nullptr, nullptr, nullptr};
            for (int l = 0; l < kk; ++l) lv[l] = seg((int)(t + 1 + l - t0));
            e = all_levels ? launch_f3_all_F32(*P, src, lv, kk, st) : cudaErrorNotSupported;
            if (e == cudaErrorNotSupported) {
                cudaGetLastError();
                for (int l = 0; l < kk; ++l) {
                    stencil_status_t s = stencil_run(P, l == 0 ? src : lv[l - 1], lv[l], 1, stream);
                    if (s != STENCIL_OK) return s;
                }
            } else if (e != cudaSuccess) {
                set_error(cudaGetErrorString(e));
                return STENCIL_ERR_CUDA;
            }
            src = lv[kk - 1];
            t += kk;
        }
        for (int64_t t = t1 - 1; t >= t0; --t) {
            p.u = static_cast<const float *>(t == t0 ? ckpt(m) : seg((int)(t - t0)));
            p.lam_in = lam_next;
            p.lam_out = static_cast<float *>(t == 0 ? grad_u0 : lam[li]);
            p.first = first ? 1 : 0;
            p.vec_ok = (P->n[2] % 4 == 0) && ((uintptr_t)p.u % 16 == 0) && ((uintptr_t)p.lam_in % 16 == 0) &&
                       ((uintptr_t)p.lam_out % 16 == 0);
            e = launch_adj(*P, p, shape, st);
            if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
            first = false;
            lam_next = p.lam_out;
            li ^= 1;
        }
    }
    adjoint_wgrad_final<<<1, 256, 0, st>>>(partials, nblocks, P->np, e2c, grad_w);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
    return STENCIL_OK;
}

}  // namespace sg

extern "C" stencil_status_t stencil_run_checkpointed(stencil_plan_t P, const void *u0, void *u_T, int64_t T,
                                                     int32_t ckpt_every, void *ckpts, void *stream) {
    if (!P || !u0 || !u_T || T < 0 || (T > ckpt_every && !ckpts)) {
        set_error("invalid argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    stencil_status_t s = adj_check(P, T, ckpt_every);
    if (s != STENCIL_OK) return s;
    if (T == 0) return stencil_run(P, u0, u_T, 0, stream);
    return forward_ckpt(P, u0, u_T, T, ckpt_every, ckpts, stream);
}

extern "C" stencil_status_t stencil_adjoint_from_checkpoints(stencil_plan_t P, const void *u0, const void *ckpts,
                                                             const void *grad_uT, int64_t T, int32_t ckpt_every,
                                                             void *grad_u0, double *grad_w, void *stream) {
    if (!P || !u0 || !grad_uT || !grad_u0 || !grad_w || T < 0 || (T > ckpt_every && !ckpts)) {
        set_error("invalid argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    stencil_status_t s = adj_check(P, T, ckpt_every);
    if (s != STENCIL_OK) return s;
    return backward_from_ckpts(P, u0, ckpts, grad_uT, T, ckpt_every, grad_u0, grad_w, stream);
}

extern "C" stencil_status_t stencil_adjoint_run(stencil_plan_t P, const void *u0, const void *grad_uT, int64_t T,
                                                int32_t ckpt_every, void *grad_u0, double *grad_w, void *stream) {
    if (!P || !u0 || !grad_uT || !grad_u0 || !grad_w || T < 0) {
        set_error("invalid argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    stencil_status_t s = adj_check(P, T, ckpt_every);
    if (s != STENCIL_OK) return s;
    if (T == 0) return backward_from_ckpts(P, u0, nullptr, grad_uT, 0, 1, grad_u0, grad_w, stream);
    // checkpoints (and a scratch u_T) in a plan-owned buffer, then the backward sweep
    const int c = ckpt_every;
    const int64_t M = (T + c - 1) / c;
    const size_t need = (size_t)M * P->grid_bytes;
    if (P->ckpt_ws_bytes < need) {
        cudaFree(P->ckpt_ws);
        P->ckpt_ws = nullptr;
        P->ckpt_ws_bytes = 0;
        if (cudaMalloc(&P->ckpt_ws, need) != cudaSuccess) {
            cudaGetLastError();
            set_error("checkpoint allocation of " + std::to_string(need) + " bytes failed");
            return STENCIL_ERR_OOM;
        }
        P->ckpt_ws_bytes = need;
    }
    void *ck = P->ckpt_ws;
    void *uT = static_cast<char *>(P->ckpt_ws) + (size_t)(M - 1) * P->grid_bytes;
    s = forward_ckpt(P, u0, uT, T, c, ck, stream);
    if (s != STENCIL_OK) return s;
    return backward_from_ckpts(P, u0, ck, grad_uT, T, c, grad_u0, grad_w, stream);
}
