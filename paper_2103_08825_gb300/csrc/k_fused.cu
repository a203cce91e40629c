// k_fused.cu -- dispatch of one fused pass (k time steps) to the kernel for
// the plan's dimension and storage type.
#include <algorithm>
#include <string>

#include "common.cuh"
#include "plan.h"

namespace sg {

#define SG_DECL_F2(DT)                                                                              \
    cudaError_t launch_f2_##DT(const stencil_plan_s &, const void *, void *, int, cudaStream_t);   \
    cudaError_t launch_f2mp_##DT(const stencil_plan_s &, const void *, void *, void *, int, int, cudaStream_t); \
    int f2_kmax_##DT(int r);                                                                        \
    int f2_bw_##DT(int r, int k);
SG_DECL_F2(F32)
SG_DECL_F2(F64)
SG_DECL_F2(BF16)
SG_DECL_F2(F16)
SG_DECL_F2(I32)
#undef SG_DECL_F2

static bool f2_multi_geom_ok(const stencil_plan_s &P, int k);

int fused2d_max_k(const stencil_plan_s &P) {
    if (P.dim != 2 || P.r > 3 || P.n[1] > (1ll << 30)) return 0;
    int km = 0;
    switch (P.dtype) {
        case STENCIL_F32: km = f2_kmax_F32(P.r); break;
        case STENCIL_F64: km = f2_kmax_F64(P.r); break;
        case STENCIL_BF16: km = f2_kmax_BF16(P.r); break;
        case STENCIL_F16: km = f2_kmax_F16(P.r); break;
        case STENCIL_I32: km = f2_kmax_I32(P.r); break;
    }
    // depths above 8 run only as the persistent kernel: the grid must allow it
    while (km > 8 && !f2_multi_geom_ok(P, km)) --km;
    return km;
}

cudaError_t launch_fused2d(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    // depths above 8 are built only as the persistent kernel: one pass of it
    if (k > 8) return launch_fused2d_multi(P, src, dst, dst, k, 1, st);
    switch (P.dtype) {
        case STENCIL_F32: return launch_f2_F32(P, src, dst, k, st);
        case STENCIL_F64: return launch_f2_F64(P, src, dst, k, st);
        case STENCIL_BF16: return launch_f2_BF16(P, src, dst, k, st);
        case STENCIL_F16: return launch_f2_F16(P, src, dst, k, st);
        case STENCIL_I32: return launch_f2_I32(P, src, dst, k, st);
    }
    return cudaErrorInvalidValue;
}

// The multi-pass kernel needs halos that wrap at most once (periodic) and
// coordinates, tiles and items that fit its 32-bit arithmetic.
bool fused2d_multi_ok(const stencil_plan_s &P, int k) {
    return P.dim == 2 && k >= 1 && k <= fused2d_max_k(P) && f2_multi_geom_ok(P, k);
}

static bool f2_multi_geom_ok(const stencil_plan_s &P, int k) {
    const int v = P.dtype == STENCIL_F64 ? 2 : 4;
    const int al = std::max(16 / (int)dtype_size(P.dtype), v);
    const int64_t h = (P.r * k + al - 1) / al * al, w = 32 * v;
    const int64_t nx = P.n[2], ny = P.n[1];
    if (nx + 2 * w >= (1ll << 30) || ny + 4 * P.r * k + 64 >= (1ll << 30)) return false;
    if (P.bkind == STENCIL_PERIODIC && (h > nx || P.r * k > ny)) return false;
    return true;
}

cudaError_t launch_fused2d_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                                 int passes, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F32: return launch_f2mp_F32(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_F64: return launch_f2mp_F64(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_BF16: return launch_f2mp_BF16(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_F16: return launch_f2mp_F16(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_I32: return launch_f2mp_I32(P, src0, dst_even, dst_odd, k, passes, st);
    }
    return cudaErrorInvalidValue;
}

std::string fused2d_describe(const stencil_plan_s &P, int k) {
    int bw = 0;
    switch (P.dtype) {
        case STENCIL_F32: bw = f2_bw_F32(P.r, k); break;
        case STENCIL_F64: bw = f2_bw_F64(P.r, k); break;
        case STENCIL_BF16: bw = f2_bw_BF16(P.r, k); break;
        case STENCIL_F16: bw = f2_bw_F16(P.r, k); break;
        case STENCIL_I32: bw = f2_bw_I32(P.r, k); break;
    }
    return "fused2d(warp-streamed rows, k=" + std::to_string(k) + ", band=" + std::to_string(bw) + " cols, tile rows=" +
           (P.tile_rows > 0 ? std::to_string(P.tile_rows) : std::string("default")) + ")";
}

#define SG_DECL_F3(DT)                                                                              \
    cudaError_t launch_f3_##DT(const stencil_plan_s &, const void *, void *, int, cudaStream_t);   \
    cudaError_t launch_f3mp_##DT(const stencil_plan_s &, const void *, void *, void *, int, int, cudaStream_t);
SG_DECL_F3(F32)
SG_DECL_F3(F64)
SG_DECL_F3(BF16)
SG_DECL_F3(F16)
SG_DECL_F3(I32)
#undef SG_DECL_F3

// 3D: k <= 4 (r = 1), 2 (r = 2 star) or 1 (r = 2 box, r = 3), bounded by
// the 2r partial planes per level each thread keeps in registers.
int fused3d_max_k(const stencil_plan_s &P) {
    if (P.dim != 3 || P.r > 3 || P.n[0] > (1ll << 30) || P.n[1] > (1ll << 30) || P.n[2] > (1ll << 30)) return 0;
    // the 125- and 343-point boxes have no fused form: one partial plane per
    // level already fills the register file, so they run the plain sweep
    if (P.pattern == STENCIL_BOX && P.r > 1) return 0;
    return P.r == 1 ? 4 : P.r == 2 ? 2 : 1;
}

cudaError_t launch_fused3d(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F32: return launch_f3_F32(P, src, dst, k, st);
        case STENCIL_F64: return launch_f3_F64(P, src, dst, k, st);
        case STENCIL_BF16: return launch_f3_BF16(P, src, dst, k, st);
        case STENCIL_F16: return launch_f3_F16(P, src, dst, k, st);
        case STENCIL_I32: return launch_f3_I32(P, src, dst, k, st);
    }
    return cudaErrorInvalidValue;
}

// As fused2d_multi_ok, for the 3D window (x halo rounded to the TMA
// alignment, y and z halos rK).
bool fused3d_multi_ok(const stencil_plan_s &P, int k) {
    if (P.dim != 3 || k < 1 || k > fused3d_max_k(P)) return false;
    const int v = P.dtype == STENCIL_F64 ? 2 : 4;
    const int al = std::max(16 / (int)dtype_size(P.dtype), v);
    const int64_t h = (P.r * k + al - 1) / al * al, rk = (int64_t)P.r * k;
    const int64_t nx = P.n[2], ny = P.n[1], nz = P.n[0];
    if (nx + 512 >= (1ll << 30) || ny + 512 >= (1ll << 30) || nz + 4 * rk + 64 >= (1ll << 30)) return false;
    if (P.bkind == STENCIL_PERIODIC && (h > nx || rk > ny || rk > nz)) return false;
    return true;
}

cudaError_t launch_fused3d_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                                 int passes, cudaStream_t st) {
    switch (P.dtype) {
        case STENCIL_F32: return launch_f3mp_F32(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_F64: return launch_f3mp_F64(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_BF16: return launch_f3mp_BF16(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_F16: return launch_f3mp_F16(P, src0, dst_even, dst_odd, k, passes, st);
        case STENCIL_I32: return launch_f3mp_I32(P, src0, dst_even, dst_odd, k, passes, st);
    }
    return cudaErrorInvalidValue;
}

bool fused_multi_ok(const stencil_plan_s &P, int k) {
    return P.dim == 1 ? fused1d_multi_ok(P, k) : P.dim == 2 ? fused2d_multi_ok(P, k) : fused3d_multi_ok(P, k);
}

cudaError_t launch_fused_multi(const stencil_plan_s &P, const void *src0, void *dst_even, void *dst_odd, int k,
                               int passes, cudaStream_t st) {
    if (P.dim == 1) return launch_fused1d_multi(P, src0, dst_even, dst_odd, k, passes, st);
    if (P.dim == 2) return launch_fused2d_multi(P, src0, dst_even, dst_odd, k, passes, st);
    if (P.dim == 3) return launch_fused3d_multi(P, src0, dst_even, dst_odd, k, passes, st);
    return cudaErrorNotSupported;
}

std::string fused3d_describe(const stencil_plan_s &P, int k) {
    return "fused3d(z-streamed planes, 64-row windows of half-warp rows, k=" + std::to_string(k) + ", planes per job=" +
           (P.tile_rows > 0 ? std::to_string(P.tile_rows) : std::string("default")) + ")";
}

int fused_max_k(const stencil_plan_s &P) {
    switch (P.dim) {
        case 1: return fused1d_max_k(P);
        case 2: return fused2d_max_k(P);
        case 3: return fused3d_max_k(P);
    }
    return 0;
}

cudaError_t launch_fused(const stencil_plan_s &P, const void *src, void *dst, int k, cudaStream_t st) {
    switch (P.dim) {
        case 1: return launch_fused1d(P, src, dst, k, st);
        case 2: return launch_fused2d(P, src, dst, k, st);
        case 3: return launch_fused3d(P, src, dst, k, st);
    }
    return cudaErrorInvalidValue;
}

std::string fused_describe(const stencil_plan_s &P, int k) {
    switch (P.dim) {
        case 1: return fused1d_describe(P, k);
        case 2: return fused2d_describe(P, k);
        case 3: return fused3d_describe(P, k);
    }
    return "none";
}

}  // namespace sg
