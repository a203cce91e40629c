// common.cuh -- shared device-side definitions of the GB300 stencil library:
// storage/compute type traits, the fixed-order multiply/FMA used by every
// kernel, compile-time stencil shapes, kernel parameter blocks and inline-PTX
// wrappers for mbarriers and TMA (cp.async.bulk.tensor) with bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/stencil.h"

namespace sg {

constexpr int kMaxPts = 343;       // box, d = 3, r = 3
constexpr int kStatusTimeout = STENCIL_ERR_TIMEOUT;

// ----------------------------------------------------------------- traits
// S: storage type in HBM; C: arithmetic type; V: elements a lane holds along
// x in the fused kernels; A: elements per 16 bytes (TMA / vector alignment).
template <int DT> struct Traits;
template <> struct Traits<STENCIL_F32> { using S = float; using C = float; static constexpr int V = 4; };
template <> struct Traits<STENCIL_F64> { using S = double; using C = double; static constexpr int V = 2; };
template <> struct Traits<STENCIL_BF16> { using S = __nv_bfloat16; using C = float; static constexpr int V = 4; };
template <> struct Traits<STENCIL_F16> { using S = __half; using C = float; static constexpr int V = 4; };
template <> struct Traits<STENCIL_I32> { using S = int32_t; using C = uint32_t; static constexpr int V = 4; };

template <int DT> constexpr int align_elems() { return 16 / (int)sizeof(typename Traits<DT>::S); }

// --------------------------------------------- fixed-order arithmetic
// Each stencil sum is mul(first term) then fma(next terms) in lexicographic
// offset order; the _rn intrinsics keep the compiler from re-contracting.
__device__ __forceinline__ float op_mul(float w, float u) { return __fmul_rn(w, u); }
__device__ __forceinline__ float op_fma(float w, float u, float a) { return __fmaf_rn(w, u, a); }
__device__ __forceinline__ double op_mul(double w, double u) { return __dmul_rn(w, u); }
__device__ __forceinline__ double op_fma(double w, double u, double a) { return __fma_rn(w, u, a); }
__device__ __forceinline__ uint32_t op_mul(uint32_t w, uint32_t u) { return w * u; }
__device__ __forceinline__ uint32_t op_fma(uint32_t w, uint32_t u, uint32_t a) { return w * u + a; }

// Row updates acc[v] (+)= w * x[v], v < V, with op_mul / op_fma (scalar:
// measured faster than the packed FP32x2 forms here, whose pair moves and
// register pressure outweighed the halved FMA count).
template <typename C, int V> __device__ __forceinline__ void row_fma_s(C w, const C *x, C *acc) {
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = op_fma(w, x[v], acc[v]);
}
template <typename C, int V> __device__ __forceinline__ void row_mul_s(C w, const C *x, C *acc) {
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = op_mul(w, x[v]);
}

// storage <-> arithmetic conversions (one rounding, to nearest even, on store)
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }
__device__ __forceinline__ uint32_t to_c(int32_t v) { return (uint32_t)v; }

template <typename S> __device__ __forceinline__ S from_c(float v);
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_c<__half>(float v) { return __float2half_rn(v); }
template <typename S> __device__ __forceinline__ S from_c(double v);
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }
template <typename S> __device__ __forceinline__ S from_c(uint32_t v);
template <> __device__ __forceinline__ int32_t from_c<int32_t>(uint32_t v) { return (int32_t)v; }

// ------------------------------------------------- stencil shapes
// Offsets are visited in lexicographic order (o_0, ..., o_{d-1}); widx gives
// the position of an included offset in that order (the index into the
// evaluation-order weight array the host prepares).
template <int D, int R, int PAT> struct Shape {
    static constexpr int npts = PAT == STENCIL_BOX ? (D == 1 ? 2 * R + 1 : D == 2 ? (2 * R + 1) * (2 * R + 1)
                                                                            : (2 * R + 1) * (2 * R + 1) * (2 * R + 1))
                                                   : 1 + 2 * D * R;
    __host__ __device__ static constexpr bool inc(int oz, int oy, int ox) {
        return PAT == STENCIL_BOX ? true : ((oz != 0) + (oy != 0) + (ox != 0)) <= 1;
    }
    // 2D (oy, ox) in-plane index, used for D == 2 and for the oz == 0 plane of D == 3
    __host__ __device__ static constexpr int widx2(int oy, int ox) {
        return PAT == STENCIL_BOX ? (oy + R) * (2 * R + 1) + (ox + R)
                                  : (oy < 0 ? oy + R : oy == 0 ? R + ox + R : R + 2 * R + 1 + oy - 1);
    }
    __host__ __device__ static constexpr int widx(int oz, int oy, int ox) {
        return D == 1 ? ox + R
             : D == 2 ? widx2(oy, ox)
             : PAT == STENCIL_BOX ? ((oz + R) * (2 * R + 1) + (oy + R)) * (2 * R + 1) + (ox + R)
                                  : (oz < 0 ? oz + R : oz == 0 ? R + widx2(oy, ox) : R + 4 * R + 1 + oz - 1);
    }
};

// --------------------------------------------------------- parameters
template <typename C> struct GridGeom {
    int64_t n0, n1, n2;   // extents padded to 3D, n0 outermost, n2 = x
    int bkind;            // STENCIL_DIRICHLET / STENCIL_PERIODIC
    C bval;
};

template <typename C> struct PlainParams {
    GridGeom<C> g;
    const void *src;
    void *dst;
    int np;                    // number of offsets (runtime-generic kernel)
    int vec_ok;                // rows 16-byte aligned (vector loads allowed)
    int off[kMaxPts][3];       // evaluation order (generic kernel only)
    C w[kMaxPts];              // evaluation (lexicographic) order
};

// ------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: gives up (returns false) after about
// `limit_ns` nanoseconds of wall time or 2^24 polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
        if (it > 32) __nanosleep(32);
    }
    return false;
}

// Wait for a copy this CTA issued before it gives up and leaves: the shared
// memory a bulk copy targets must outlive the copy.  Up to about ten seconds
// (ten bounded waits); false if the copy still had not landed.
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < 10; ++i)
        if (mbar_wait_bounded(bar, parity)) return true;
    return false;
}

// 2D / 3D tiled TMA loads (global -> shared), completion on an mbarrier.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void record_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------- cross-CTA completion counters
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Job tickets of the one-launch-per-pass kernels (16 bytes of the plan's
// status block).
struct JobCtl {
    unsigned long long ticket;
    unsigned exited;   // workers (warps or CTAs) that have left the launch
    unsigned pad;
};
static_assert(sizeof(JobCtl) == 16, "job tickets occupy 16 bytes of the plan's status block");

// A launch leaves its counters clean for the next launch -- also when a
// captured CUDA graph replays the same launch with the same parameters:
// every worker counts itself out after its last access, and the one that
// finds itself last (true here) resets what the launch used.  Called by one
// thread per worker.
__device__ __forceinline__ bool worker_exit_is_last(unsigned *exited, unsigned workers) {
    __threadfence();
    const bool last = atomicAdd(exited, 1u) == workers - 1;
    if (last) __threadfence();
    return last;
}

// *ctr += v with release semantics at GPU scope: this thread's earlier
// accesses (and those it has observed, e.g. through __syncwarp) are visible
// to any thread that acquires the new value
__device__ __forceinline__ void red_release_add(int *ctr, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(ctr), "r"(v) : "memory");
}

// orders this thread's generic-proxy global accesses with its async-proxy
// (TMA) ones: taken after acquiring data that other CTAs stored and before
// reading it by TMA, and after storing data that other CTAs will read by TMA
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Wait until *ctr >= target (acquire), the abort flag rises, or about one
// second of wall time passes; false unless the target was reached.
__device__ __forceinline__ bool wait_counter(const int *ctr, int target, const int *abort_flag) {
    if (ld_acquire(ctr) >= target) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (ld_acquire(ctr) >= target) return true;
        if (ld_relaxed(abort_flag)) return false;
        if (global_ns() - t0 > 1000000000ull) return false;
        __nanosleep(it < 16 ? 32 : 256);
    }
    return false;
}

// The tiles along one axis (tile t covers [t len, min((t+1) len, n))) whose
// range meets the coordinate range [lo, hi): the clipped range, plus for a
// periodic axis its images wrapped from below and above.  Three intervals of
// tile indices, some possibly empty or overlapping; requires -n <= lo and
// hi <= 2n.
struct TileSpan {
    int a0, n0, a1, n1, a2, n2;
    __host__ __device__ __forceinline__ int count() const { return n0 + n1 + n2; }
    __host__ __device__ __forceinline__ int at(int i) const {
        return i < n0 ? a0 + i : i < n0 + n1 ? a1 + i - n0 : a2 + i - n0 - n1;
    }
};

__host__ __device__ __forceinline__ TileSpan tile_span(int lo, int hi, int n, int len, bool periodic) {
    TileSpan s{0, 0, 0, 0, 0, 0};
    const int c0 = lo > 0 ? lo : 0, c1 = hi < n ? hi : n;
    if (c0 < c1) { s.a0 = c0 / len; s.n0 = (c1 - 1) / len + 1 - s.a0; }
    if (periodic && lo < 0) {   // [lo, min(hi, 0)) wrapped up by n
        const int w1 = (hi < 0 ? hi : 0) + n;
        s.a1 = (lo + n) / len;
        s.n1 = (w1 - 1) / len + 1 - s.a1;
    }
    if (periodic && hi > n) {   // [max(lo, n), hi) wrapped down by n
        const int w0 = (lo > n ? lo : n) - n;
        s.a2 = w0 / len;
        s.n2 = (hi - n - 1) / len + 1 - s.a2;
    }
    return s;
}

__host__ __device__ constexpr int round_up_c(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ constexpr int max_c(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
__host__ __device__ constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// 16-byte global -> shared copies (L2 only), grouped and waited for per group
__device__ __forceinline__ void cp_async16(void *smem, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ int64_t wrap_idx(int64_t i, int64_t n) {
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

}  // namespace sg
