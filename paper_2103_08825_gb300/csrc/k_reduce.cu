// k_reduce.cu -- FP64 reductions over a grid: sum (mass), sum of squares,
// and the loss 0.5 * ||u - target||^2.  Elements are widened to FP64 exactly
// and summed in an order fixed by n alone (block b owns a contiguous range,
// thread t a stride of it, then a fixed tree), so results do not depend on
// the device or on timing.  Two passes: per-block partials, then one block.
#include <mutex>
#include <string>

#include "common.cuh"
#include "plan.h"

namespace sg {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
__device__ __forceinline__ double widen(__half v) { return (double)__half2float(v); }

__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + s];
        __syncthreads();
    }
    return sh[0];
}

template <typename S, int OP>
__global__ void __launch_bounds__(RED_THREADS)
    reduce_partials(const S *__restrict__ u, const S *__restrict__ tg, int64_t n, int64_t per_block, double *part) {
    __shared__ double sh[RED_THREADS];
    const int64_t lo = (int64_t)blockIdx.x * per_block;
    const int64_t hi = lo + per_block < n ? lo + per_block : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += RED_THREADS) {
        const double x = widen(u[i]);
        if (OP == STENCIL_REDUCE_SUM) acc = acc + x;
        else if (OP == STENCIL_REDUCE_SUMSQ) acc = __fma_rn(x, x, acc);
        else {
            const double e = x - widen(tg[i]);
            acc = __fma_rn(e, e, acc);
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <int OP>
__global__ void __launch_bounds__(RED_THREADS) reduce_final(const double *__restrict__ part, int nb, double *out) {
    __shared__ double sh[RED_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += RED_THREADS) acc = acc + part[i];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = (OP == STENCIL_REDUCE_HALF_SQDIST) ? 0.5 * s : s;
}

// Launch both passes with `part` (>= reduce_blocks(n) doubles) as scratch.
template <typename S>
static cudaError_t reduce_launch_t(int64_t n, const void *u, const void *tg, int op, double *part, double *out,
                                   cudaStream_t st, int nb, int64_t per) {
    const S *pu = static_cast<const S *>(u);
    const S *pt = static_cast<const S *>(tg);
    switch (op) {
        case STENCIL_REDUCE_SUM:
            reduce_partials<S, STENCIL_REDUCE_SUM><<<nb, RED_THREADS, 0, st>>>(pu, pt, n, per, part);
            reduce_final<STENCIL_REDUCE_SUM><<<1, RED_THREADS, 0, st>>>(part, nb, out);
            break;
        case STENCIL_REDUCE_SUMSQ:
            reduce_partials<S, STENCIL_REDUCE_SUMSQ><<<nb, RED_THREADS, 0, st>>>(pu, pt, n, per, part);
            reduce_final<STENCIL_REDUCE_SUMSQ><<<1, RED_THREADS, 0, st>>>(part, nb, out);
            break;
        default:
            reduce_partials<S, STENCIL_REDUCE_HALF_SQDIST><<<nb, RED_THREADS, 0, st>>>(pu, pt, n, per, part);
            reduce_final<STENCIL_REDUCE_HALF_SQDIST><<<1, RED_THREADS, 0, st>>>(part, nb, out);
    }
    return cudaGetLastError();
}

int reduce_blocks(int64_t n) {
    int64_t nb = (n + 4095) / 4096;
    if (nb < 1) nb = 1;
    if (nb > RED_MAX_BLOCKS) nb = RED_MAX_BLOCKS;   // the partial-sum buffers hold RED_MAX_BLOCKS doubles
    return (int)nb;
}

cudaError_t reduce_launch(int dtype, int64_t n, const void *u, const void *tg, int op, double *part, double *out,
                          cudaStream_t st) {
    const int nb = reduce_blocks(n);
    const int64_t per = (n + nb - 1) / nb;
    switch (dtype) {
        case STENCIL_F64: return reduce_launch_t<double>(n, u, tg, op, part, out, st, nb, per);
        case STENCIL_F32: return reduce_launch_t<float>(n, u, tg, op, part, out, st, nb, per);
        case STENCIL_BF16: return reduce_launch_t<__nv_bfloat16>(n, u, tg, op, part, out, st, nb, per);
        case STENCIL_F16: return reduce_launch_t<__half>(n, u, tg, op, part, out, st, nb, per);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sg

using namespace sg;

extern "C" stencil_status_t stencil_reduce(int32_t dtype, int64_t n, const void *u, const void *target, int32_t op,
                                           double *out, void *stream) {
    if (dtype == STENCIL_I32 || dtype < STENCIL_F64 || dtype > STENCIL_F16) {
        set_error("stencil_reduce supports F64, F32, BF16 and F16");
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (n < 1 || !u || !out || op < STENCIL_REDUCE_SUM || op > STENCIL_REDUCE_HALF_SQDIST ||
        (op == STENCIL_REDUCE_HALF_SQDIST && !target)) {
        set_error("invalid reduction arguments");
        return STENCIL_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *part = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&part), sizeof(double) * reduce_blocks(n), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("partial-sum allocation failed");
        return STENCIL_ERR_OOM;
    }
    e = reduce_launch(dtype, n, u, target, op, part, out, st);
    cudaError_t e2 = cudaFreeAsync(part, st);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        set_error(std::string("reduction launch: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        return STENCIL_ERR_CUDA;
    }
    return STENCIL_OK;
}

// ------------------------------------------------------------------------
// Allocation-free variant.  The partial sums of the first pass live in this
// file-scope device array instead of a stream-ordered allocation.  Its size
// is the largest number of partials the reduction ever uses (reduce_blocks
// clamps the partition to RED_MAX_BLOCKS, 8 KiB of doubles), and every GPU
// that loads the library keeps it until the process exits.  Host code must
// not hand the array's host-side name to a kernel: its device address is
// looked up with cudaGetSymbolAddress, with the device current, and cached
// together with the context it belongs to; a call made under another context
// of the same device (after cudaDeviceReset, say) looks it up again.
static __device__ __align__(256) double g_reduce_scratch[RED_MAX_BLOCKS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
struct ScratchAddr {
    double *addr;
    void *ctx;
};
ScratchAddr g_scratch[kMaxDevices] = {};

typedef int (*CtxGetCurrentFn)(void **);

// The driver's cuCtxGetCurrent, through the runtime's entry-point query (the
// library does not link libcuda directly).  Null if unavailable.
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}
}  // namespace

extern "C" stencil_status_t stencil_reduce_noalloc(int32_t dtype, int64_t n, const void *u, const void *target,
                                                   int32_t op, double *out, void *stream) {
    if (dtype == STENCIL_I32 || dtype < STENCIL_F64 || dtype > STENCIL_F16) {
        set_error("stencil_reduce_noalloc supports F64, F32, BF16 and F16");
        return STENCIL_ERR_UNSUPPORTED;
    }
    if (n < 1 || !u || !out || op < STENCIL_REDUCE_SUM || op > STENCIL_REDUCE_HALF_SQDIST ||
        (op == STENCIL_REDUCE_HALF_SQDIST && !target)) {
        set_error("invalid reduction arguments");
        return STENCIL_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_error("stencil_reduce_noalloc: no usable current device");
        return STENCIL_ERR_CUDA;
    }
    // make the device's primary context current (CUDA 12 and later initialise
    // it here; a no-op when it already is), so that the context handle below
    // names the one the launch will use
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        set_error(std::string("stencil_reduce_noalloc: cudaSetDevice failed: ") + cudaGetErrorString(e));
        return STENCIL_ERR_CUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        void *ctx = nullptr;
        if (CtxGetCurrentFn f = ctx_get_current()) f(&ctx);
        ScratchAddr &s = g_scratch[dev];
        if (!s.addr || s.ctx != ctx) {
            // first call on this device (or in a new context): find the array's device address
            double *a = nullptr;
            e = cudaGetSymbolAddress(reinterpret_cast<void **>(&a), g_reduce_scratch);
            if (e != cudaSuccess) {
                s.addr = nullptr;
                set_error(std::string("stencil_reduce_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
                return STENCIL_ERR_CUDA;
            }
            s.addr = a;
            s.ctx = ctx;
        }
        scratch = s.addr;
    }
    // every partial slot the final pass reads is written by the first pass
    // of the same call (reduce_blocks(n) <= RED_MAX_BLOCKS slots), so nothing
    // needs clearing
    e = reduce_launch(dtype, n, u, target, op, scratch, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_error(std::string("reduction launch: ") + cudaGetErrorString(e));
        return STENCIL_ERR_CUDA;
    }
    return STENCIL_OK;
}
