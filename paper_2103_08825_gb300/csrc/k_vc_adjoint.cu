// k_vc_adjoint.cu -- reverse-mode derivative of the variable-coefficient
// sweep u_{t+1}[x] = sum_o c_o[x] u_t(x + o) (FP32 and FP64 plans, d = 1..3).
//
// Not in the paper (neither the coefficient fields nor the derivative are).
// For a loss L(u_T) with lam_T = dL/du_T, walking t = T-1 .. 0:
//     dL/dc_o[x] += lam_{t+1}[x] * u_t(x + o)          (the boundary value where
//                                                      x + o lies outside a Dirichlet domain)
//     lam_t[y]    = sum_o c_o[y - o] * lam_{t+1}[y - o] (y - o wrapped on periodic
//                                                      axes, dropped outside a Dirichlet domain)
// and dL/du_0 = lam_0.  One kernel does both lines of a step for 4 points of
// a row per thread; the coefficient gradient is accumulated in place in the
// arithmetic type, the offsets taken from the plan at run time (as the
// one-step forward kernel).  Forward states: checkpoints every c steps taken
// by a forward sweep of stencil_run_vc, each segment's inner states
// recomputed one step per launch.
#include <algorithm>
#include <string>

#include "k_vc.cuh"

namespace sg {

template <typename C> struct VcAdjParams {
    const C *lam_in;        // lam_{t+1}
    const C *u;             // u_t
    const C *coef;          // [np][N], compact order
    C *lam_out;             // lam_t
    C *gcoef;               // [np][N]
    int64_t N, n0, n1, n2;
    int bkind;
    C bval;
    int np;
    int first;              // 1: overwrite gcoef, 0: add
    short ci[kMaxPts];
    signed char off[kMaxPts][3];
};

// index of (i0, i1, i2) after wrapping (periodic) or -1 outside a Dirichlet domain
__device__ __forceinline__ int64_t vca_resolve(int64_t i0, int64_t i1, int64_t i2, int64_t n0, int64_t n1,
                                               int64_t n2, bool periodic) {
    if (i0 < 0 || i0 >= n0) { if (!periodic) return -1; i0 = wrap_idx(i0, n0); }
    if (i1 < 0 || i1 >= n1) { if (!periodic) return -1; i1 = wrap_idx(i1, n1); }
    if (i2 < 0 || i2 >= n2) { if (!periodic) return -1; i2 = wrap_idx(i2, n2); }
    return (i0 * n1 + i1) * n2 + i2;
}

template <typename C>
__global__ void __launch_bounds__(256) vc_adjoint_kernel(const __grid_constant__ VcAdjParams<C> p) {
    constexpr int VX = 4;
    const bool periodic = p.bkind == STENCIL_PERIODIC;
    const int64_t n0 = p.n0, n1 = p.n1, n2 = p.n2;
    const int64_t groups = (n2 + VX - 1) / VX;
    const int64_t items = n0 * n1 * groups;
    for (int64_t it = blockIdx.x * 256ll + threadIdx.x; it < items; it += (int64_t)gridDim.x * 256) {
        const int64_t g = it % groups, row = it / groups;
        const int64_t i1 = row % n1, i0 = row / n1;
#pragma unroll
        for (int v = 0; v < VX; ++v) {
            const int64_t i2 = g * VX + v;
            if (i2 >= n2) break;
            const int64_t y = (i0 * n1 + i1) * n2 + i2;
            const C ly = p.lam_in[y];
            C acc = C(0);
#pragma unroll 1
            for (int j = 0; j < p.np; ++j) {
                const int o0 = p.off[j][0], o1 = p.off[j][1], o2 = p.off[j][2];
                const int64_t cj = (int64_t)p.ci[j] * p.N;
                // lam_t[y] gathers c_o[x] lam[x] from the x with x + o = y
                const int64_t x = vca_resolve(i0 - o0, i1 - o1, i2 - o2, n0, n1, n2, periodic);
                if (x >= 0) acc = op_fma(p.coef[cj + x], p.lam_in[x], acc);
                // dL/dc_o[y] += lam[y] u(y + o)
                const int64_t yo = vca_resolve(i0 + o0, i1 + o1, i2 + o2, n0, n1, n2, periodic);
                const C uv = yo >= 0 ? p.u[yo] : p.bval;
                C *gp = p.gcoef + cj + y;
                *gp = p.first ? op_mul(ly, uv) : op_fma(ly, uv, *gp);
            }
            p.lam_out[y] = acc;
        }
    }
}

template <typename C>
static cudaError_t launch_vc_adj(const stencil_plan_s &P, const void *lam_in, const void *u, const void *coef,
                                 void *lam_out, void *gcoef, bool first, cudaStream_t st) {
    VcAdjParams<C> p;
    p.lam_in = static_cast<const C *>(lam_in);
    p.u = static_cast<const C *>(u);
    p.coef = static_cast<const C *>(coef);
    p.lam_out = static_cast<C *>(lam_out);
    p.gcoef = static_cast<C *>(gcoef);
    p.N = P.npts;
    p.n0 = P.n[0];
    p.n1 = P.n[1];
    p.n2 = P.n[2];
    p.bkind = P.bkind;
    p.bval = (C)P.bval;
    p.np = P.np;
    p.first = first ? 1 : 0;
    for (int j = 0; j < P.np; ++j) {
        p.ci[j] = (short)P.eval_to_compact[j];
        for (int a = 0; a < 3; ++a) p.off[j][a] = (signed char)P.off_eval[j][a];
    }
    const int64_t items = P.n[0] * P.n[1] * ((P.n[2] + 3) / 4);
    int64_t blocks = (items + 255) / 256;
    if (blocks > (int64_t)P.sm_count * 16) blocks = (int64_t)P.sm_count * 16;
    vc_adjoint_kernel<C><<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace sg

using namespace sg;

extern "C" stencil_status_t stencil_adjoint_vc(stencil_plan_t P, const void *coef, const void *u0,
                                               const void *grad_uT, int64_t T, int32_t ckpt_every, void *grad_u0,
                                               void *grad_coef, void *stream) {
    if (!P || !coef || !u0 || !grad_uT || !grad_u0 || !grad_coef || T < 0) {
        set_error("invalid argument");
        return STENCIL_ERR_INVALID_ARG;
    }
    if (P->dtype != STENCIL_F32 && P->dtype != STENCIL_F64) {
        set_error("the variable-coefficient adjoint supports F32 and F64 plans");
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (T > 0 && (ckpt_every < 1 || ckpt_every > T)) {
        set_error("ckpt_every must be in 1..T");
        return STENCIL_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t gb = P->grid_bytes, cbytes = gb * (size_t)P->np;
    if (T == 0) {
        cudaError_t e = cudaMemcpyAsync(grad_u0, grad_uT, gb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(grad_coef, 0, cbytes, st);
        return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cudaMemcpyAsync");
    }
    const int c = ckpt_every;
    const int64_t M = (T + c - 1) / c;
    // workspace: checkpoints after c, 2c, .., (M - 1) c steps; c - 1 segment
    // states; two lam grids
    const size_t ngrids = (size_t)(M - 1) + (size_t)(c - 1) + 2;
    if (P->vcadj_ws_bytes < ngrids * gb) {
        cudaFree(P->vcadj_ws);
        P->vcadj_ws = nullptr;
        P->vcadj_ws_bytes = 0;
        if (cudaMalloc(&P->vcadj_ws, ngrids * gb) != cudaSuccess) {
            cudaGetLastError();
            set_error("variable-coefficient adjoint workspace allocation of " + std::to_string(ngrids * gb) +
                      " bytes failed");
            return STENCIL_ERR_OOM;
        }
        P->vcadj_ws_bytes = ngrids * gb;
    }
    char *ws = static_cast<char *>(P->vcadj_ws);
    auto grid_at = [&](size_t i) { return static_cast<void *>(ws + i * gb); };
    auto ckpt = [&](int64_t m) -> const void * { return m == 0 ? u0 : grid_at((size_t)(m - 1)); };
    auto seg = [&](int64_t i) { return grid_at((size_t)(M - 1) + (size_t)(i - 1)); };   // i = 1 .. c - 1
    void *lam[2] = {grid_at((size_t)(M - 1) + (size_t)(c - 1)), grid_at((size_t)(M - 1) + (size_t)c)};
    // forward: the checkpoints
    for (int64_t m = 1; m < M; ++m) {
        stencil_status_t s = stencil_run_vc(P, coef, ckpt(m - 1), grid_at((size_t)(m - 1)), c, stream);
        if (s != STENCIL_OK) return s;
    }
    // backward, segment by segment
    const void *lam_next = grad_uT;
    int li = 0;
    bool first = true;
    for (int64_t m = M - 1; m >= 0; --m) {
        const int64_t t0 = m * c, t1 = std::min<int64_t>(T, t0 + c);
        for (int64_t t = t0 + 1; t < t1; ++t) {
            stencil_status_t s = stencil_run_vc(P, coef, t - 1 == t0 ? ckpt(m) : seg(t - 1 - t0), seg(t - t0), 1,
                                                stream);
            if (s != STENCIL_OK) return s;
        }
        for (int64_t t = t1 - 1; t >= t0; --t) {
            const void *u = t == t0 ? ckpt(m) : seg(t - t0);
            void *out = t == 0 ? grad_u0 : lam[li];
            cudaError_t e = P->dtype == STENCIL_F64
                                ? launch_vc_adj<double>(*P, lam_next, u, coef, out, grad_coef, first, st)
                                : launch_vc_adj<float>(*P, lam_next, u, coef, out, grad_coef, first, st);
            if (e != cudaSuccess) return cuda_fail(e, "variable-coefficient adjoint launch");
            first = false;
            lam_next = out;
            li ^= 1;
        }
    }
    return STENCIL_OK;
}
