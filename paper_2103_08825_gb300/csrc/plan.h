// plan.h -- host-side plan object and the internal launch interface between
// the C ABI (api.cu) and the kernel translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/stencil.h"

namespace sg {
constexpr int kHostMaxPts = 343;
constexpr size_t kMpCtlBytes = 16;   // the control block of a persistent multi-pass launch
}

struct stencil_plan_s {
    int dim = 0, r = 0, pattern = 0, np = 0, dtype = 0, bkind = 0;
    double bval = 0.0;
    int64_t n[3] = {1, 1, 1};   // padded to 3D: n[0] outermost, n[2] unit stride
    int64_t npts = 0;
    double w_compact[sg::kHostMaxPts] = {};
    // evaluation (lexicographic) order of the offsets and their weights
    int off_eval[sg::kHostMaxPts][3] = {};
    double w_eval[sg::kHostMaxPts] = {};
    int eval_to_compact[sg::kHostMaxPts] = {};
    int k = 0;                 // 0 = default
    int tile_rows = 0;         // 2D fused tile height (0 = default)
    int block_warps = 0;       // 2D fused kernels: warps per CTA (0 = default 4)
    int variant = STENCIL_VARIANT_FUSED;
    bool tuned_plain = false;  // the tuner found the one-step kernel fastest
    int device = 0;
    int sm_count = 0;
    void *ws = nullptr;        // one grid: intermediate passes of stencil_run
    void *hws[2] = {nullptr, nullptr};   // device copies for stencil_run_host
    // stencil_run_host_many: two input and two output grids, copy streams, events
    void *hm_buf[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t hm_st[2] = {nullptr, nullptr};
    cudaEvent_t hm_ev[7] = {};
    bool hm_ready = false;
    size_t grid_bytes = 0;
    int *d_status = nullptr;   // device status word (0 = OK)
    void *d_ctr = nullptr;     // job tickets of the per-pass kernels (sg::JobCtl, same allocation)
    // persistent multi-pass launches: a control block, then one pass counter
    // per tile; every launch leaves them at zero
    mutable void *d_mp = nullptr;
    mutable int64_t mp_tiles_cap = 0;
    // in-place sweep: two ring buffers
    void *inpl_ws = nullptr;
    size_t inpl_ws_bytes = 0;
    // adjoint: plan-owned checkpoints (stencil_adjoint_run) and workspace
    void *ckpt_ws = nullptr;
    size_t ckpt_ws_bytes = 0;
    void *adj_ws = nullptr;
    size_t adj_ws_bytes = 0;
    void *vcadj_ws = nullptr;   // variable-coefficient adjoint: checkpoints, segment states, lam grids
    size_t vcadj_ws_bytes = 0;
    double *adj_partials = nullptr;
    size_t adj_partials_n = 0;
};

namespace sg {

size_t dtype_size(int dtype);

// one plain Jacobi step: dst = A(src)   (k_plain.cu)
cudaError_t launch_plain(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st);

// one fused pass of `k` steps (k_fused1d.cu / k_fused2d_*.cu / k_fused3d.cu)
int fused_max_k(const stencil_plan_s &P);
cudaError_t launch_fused(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st);
std::string fused_describe(const stencil_plan_s &P, int k);

// per-dimension entry points used by launch_fused
int fused2d_max_k(const stencil_plan_s &P);
cudaError_t launch_fused2d(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st);
// `passes` passes of k steps in one persistent launch: pass 0 reads src0, the
// passes p with (passes - 1 - p) even write dst_even, the others dst_odd.
// cudaErrorNotSupported when the geometry needs one launch per pass.
cudaError_t launch_fused2d_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                                 int passes, cudaStream_t st);
bool fused2d_multi_ok(const stencil_plan_s &P, int k);
bool fused3d_multi_ok(const stencil_plan_s &P, int k);
bool fused1d_multi_ok(const stencil_plan_s &P, int k);
cudaError_t launch_fused1d_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                                 int passes, cudaStream_t st);
cudaError_t launch_fused3d_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                                 int passes, cudaStream_t st);
// the persistent multi-pass form for the plan's dimension
bool fused_multi_ok(const stencil_plan_s &P, int k);
cudaError_t launch_fused_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                               int passes, cudaStream_t st);
// control state of the persistent launches for `tiles` tiles (grown on demand)
cudaError_t ensure_mp_state(const stencil_plan_s &P, int64_t tiles, cudaStream_t st);
std::string fused2d_describe(const stencil_plan_s &P, int k);
int fused3d_max_k(const stencil_plan_s &P);
// one 3D FP32 radius-1 pass of k <= 4 steps storing every level (lv[l - 1] = level l)
cudaError_t launch_f3_all_F32(const stencil_plan_s &P, const void *src, void *const *lv, int k, cudaStream_t st);
cudaError_t launch_fused3d(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st);
std::string fused3d_describe(const stencil_plan_s &P, int k);
int fused1d_max_k(const stencil_plan_s &P);
cudaError_t launch_fused1d(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st);
std::string fused1d_describe(const stencil_plan_s &P, int k);

// TMA descriptor for a dense row-major grid (box dims innermost first)
bool make_tmap(CUtensorMap *map, int dtype, int rank, const int64_t *dims_inner_first, const uint32_t *box,
               const void *base);

void set_error(const std::string &msg);
stencil_status_t cuda_fail(cudaError_t e, const char *what);
stencil_status_t ensure_buf(void **buf, size_t bytes);
stencil_status_t ensure_status_word(stencil_plan_s *P);
// T steps by tessellate tiling (k_tess.cu)
stencil_status_t tess_run(stencil_plan_s *P, const void *u_in, void *u_out, int64_t T, cudaStream_t st);

}  // namespace sg
