// k_batch.cu -- many independent 2D grids advanced by one persistent kernel.
//
// Not in the paper (which runs one grid at a time): grids of uneven size and
// step count share the GPU through a work queue.  Each grid's passes (k
// fused steps; the first one the remainder T - (passes - 1) k, so that only
// pass 0 mixes fusion depths -- and instruction streams -- across grids,
// the result being the same for any grouping of the steps) are cut into
// warp-sized tiles (one
// column band x Ly rows).  Items (grid, pass, tile) are listed pass-major;
// worker warps take the next item from an atomic ticket, wait until every
// tile whose output meets the item's input window (wrapped for periodic
// grids; listed on the host per column band and per row chunk) has finished
// the previous pass -- exactly the tiles whose outputs it reads and whose
// inputs its output overwrites -- then run the same warp-streamed
// fused job as stencil_run and publish completion.  Because every
// dependency precedes the item in the queue and all workers are resident,
// the waits always end; they are still bounded (about one second of
// wall time), and one that gives up raises an abort flag that stops every
// worker and sets the batch's status word to STENCIL_ERR_TIMEOUT.
//
// The kernel plus the counter resets are captured into a CUDA graph on the
// first stencil_batch_run and replayed afterwards.
#include <string.h>

#include <cmath>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "k_fused2d.cuh"
#include "plan.h"

namespace sg {

constexpr int BT_NW = 4;          // warps per CTA
constexpr int BT_LY = 64;         // default output rows per tile (stencil_batch_set_config)
constexpr int BT_MAXW = 25;

template <typename C> struct BatchGrid {
    const void *in;
    void *out;
    void *ws;
    int ny, nx;
    int passes, k_first;   // the first pass advances k_first <= KB steps, the others KB
    int bands, chunks;
    int tile_base;       // index of this grid's first tile counter
    int boff, coff;      // this grid's band / chunk offsets into dep_off
    C w[BT_MAXW];        // evaluation order
};

struct BatchCtl {
    unsigned long long ticket;
    int abort;
    int status;
};

template <typename C> struct BatchParams {
    const BatchGrid<C> *grids;
    const unsigned long long *items;   // grid | pass << 16 | tile << 32
    long long nitems;
    int *done;                         // passes finished, per tile
    const int *dep_off;                // per band / chunk: range of its dependency list
    const int *dep_list;               // bands (chunks) whose outputs meet its input window
    BatchCtl *ctl;
    int bkind;
    int ly;                            // output rows per tile
    C bval;
    int *test_skip_publish;            // test hook: never publish this item (host-side fault injection)
};

template <int DT, int R, int PAT, int K, int KB, bool MASK>
__device__ __forceinline__ void batch_job(const BatchGrid<typename Traits<DT>::C> &G, const void *src, void *dst,
                                          bool dir, typename Traits<DT>::C bval,
                                          const typename Traits<DT>::C *wr, int64_t xo0, int64_t yo0, int64_t yo1,
                                          bool vec_ok, uint32_t &gst, int lane) {
    using S = typename Traits<DT>::S;
    // tiles are cut with k = KB's band width; a shorter first pass must write
    // exactly the same columns
    static_assert(F2Geo<DT, R, K>::BW == F2Geo<DT, R, KB>::BW, "band width must not depend on k <= KB");
    fused2d_job<DT, R, PAT, K, PROD_REG, true, MASK>(nullptr, static_cast<const S *>(src), static_cast<S *>(dst),
                                                     G.nx, G.ny, dir, bval, wr, xo0, yo0, yo1, vec_ok, nullptr,
                                                     nullptr, gst, lane);
}

template <int DT, int R, int PAT, int KB>
__global__ void __launch_bounds__(BT_NW * 32) batch_kernel(const __grid_constant__ BatchParams<typename Traits<DT>::C> p) {
    using C = typename Traits<DT>::C;
    using Sh = Shape<2, R, PAT>;
    const int lane = threadIdx.x & 31;
    const bool dir = p.bkind == STENCIL_DIRICHLET;
    uint32_t gst = 0;
    while (true) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(&p.ctl->ticket, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((long long)q >= p.nitems) break;
        if (__shfl_sync(0xffffffffu, lane == 0 ? ld_relaxed(&p.ctl->abort) : 0, 0)) break;
        const unsigned long long item = p.items[q];
        const int g = (int)(item & 0xffffull), pass = (int)((item >> 16) & 0xffffull), t = (int)(item >> 32);
        const BatchGrid<C> &G = p.grids[g];
        const int b = t % G.bands, c = t / G.bands;
        // dependencies: every tile of the previous pass whose output meets
        // this tile's input window (= whose input window meets its output)
        bool ok = true;
        if (pass > 0) {
            const int b0 = p.dep_off[G.boff + b], nbx = p.dep_off[G.boff + b + 1] - b0;
            const int c0 = p.dep_off[G.coff + c], ncy = p.dep_off[G.coff + c + 1] - c0;
            for (int e = lane; e < nbx * ncy; e += 32) {
                const int nb = p.dep_list[b0 + e % nbx], nc = p.dep_list[c0 + e / nbx];
                ok = ok && wait_counter(&p.done[G.tile_base + nc * G.bands + nb], pass, &p.ctl->abort);
            }
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicExch(&p.ctl->abort, 1);
                atomicCAS(&p.ctl->status, 0, kStatusTimeout);
            }
            break;
        }
        __threadfence();
        // buffers: the last pass writes `out`, earlier ones alternate ws / out
        const void *src = pass == 0 ? G.in : (((G.passes - pass) % 2 == 0) ? G.out : G.ws);
        void *dst = ((G.passes - 1 - pass) % 2 == 0) ? G.out : G.ws;
        const int kp = pass == 0 ? G.k_first : KB;
        C wr[Sh::npts];
#pragma unroll
        for (int j = 0; j < Sh::npts; ++j) wr[j] = G.w[j];
        using Geo = F2Geo<DT, R, KB>;
        const int64_t xo0 = (int64_t)b * Geo::BW;
        const int64_t yo0 = (int64_t)c * p.ly;
        const int64_t yo1 = yo0 + p.ly < G.ny ? yo0 + p.ly : G.ny;
        const bool vec_ok = (G.nx % Traits<DT>::V == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
        // tiles are laid out with the band width of k = KB; shorter first
        // passes use the same tiles (their halo is smaller)
        const bool interior = !dir || (xo0 - Geo::H >= 0 && xo0 - Geo::H + Geo::W <= G.nx && yo0 - R * KB >= 0 &&
                                       yo1 + R * KB <= G.ny);
#define SG_BJ(KK)                                                                                           \
    if (interior) batch_job<DT, R, PAT, KK, KB, false>(G, src, dst, dir, p.bval, wr, xo0, yo0, yo1, vec_ok, gst, lane); \
    else batch_job<DT, R, PAT, KK, KB, true>(G, src, dst, dir, p.bval, wr, xo0, yo0, yo1, vec_ok, gst, lane);
        switch (kp) {
            case 1: { SG_BJ(1) break; }
            case 2: { if constexpr (KB >= 2) { SG_BJ(2) } break; }
            case 3: { if constexpr (KB >= 3) { SG_BJ(3) } break; }
            case 4: { if constexpr (KB >= 4) { SG_BJ(4) } break; }
        }
#undef SG_BJ
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            if (!(p.test_skip_publish && *p.test_skip_publish == (int)q)) atomicAdd(&p.done[G.tile_base + t], 1);
        }
    }
}

}  // namespace sg

using namespace sg;

struct stencil_batch_s {
    int n = 0, r = 0, pattern = 0, dtype = 0, bkind = 0, kb = 4, ly = BT_LY;
    double bval = 0.0;
    int device = 0, sm_count = 0;
    std::vector<int64_t> ny, nx, T;
    std::vector<double> wts;          // every member's compact weights (schedule rebuilds)
    int np = 0;
    std::vector<size_t> bytes;
    void *d_grids = nullptr;          // BatchGrid<C>[n]
    std::vector<unsigned char> h_grids;
    size_t grid_desc_size = 0;
    unsigned long long *d_items = nullptr;
    int *d_dep_off = nullptr, *d_dep_list = nullptr;
    long long nitems = 0;
    int *d_done = nullptr;
    long long ntiles = 0;
    BatchCtl *d_ctl = nullptr;
    int *d_skip = nullptr;            // test hook (fault injection), null unless enabled
    std::vector<void *> ws;
    std::vector<const void *> last_in;
    std::vector<void *> last_out;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid_ctas = 0;
};

namespace {

int tile_bw(int dtype, int r, int kb) {
    // band width of the 2D fused job for (dtype, r, k = kb)
    const int v = dtype == STENCIL_F64 ? 2 : 4;
    const int al = std::max(16 / (int)dtype_size(dtype), v);
    const int h = (r * kb + al - 1) / al * al;
    return 32 * v - 2 * h;
}

template <int DT>
stencil_status_t build_batch(stencil_batch_s *B);

template <int DT>
stencil_status_t rebuild_batch(stencil_batch_s *B) { return build_batch<DT>(B); }

template <int DT>
stencil_status_t build_batch(stencil_batch_s *B) {
    using C = typename Traits<DT>::C;
    const int n = B->n;
    B->grid_desc_size = sizeof(BatchGrid<C>);
    B->h_grids.assign(sizeof(BatchGrid<C>) * n, 0);
    BatchGrid<C> *hg = reinterpret_cast<BatchGrid<C> *>(B->h_grids.data());
    const int bw = tile_bw(DT, B->r, B->kb);
    // evaluation (lexicographic) order of the compact 2D weights
    const int np = B->pattern == STENCIL_BOX ? (2 * B->r + 1) * (2 * B->r + 1) : 1 + 4 * B->r;
    std::vector<std::pair<int, int>> offs(np);
    if (B->pattern == STENCIL_BOX) {
        for (int j = 0; j < np; ++j) offs[j] = {j / (2 * B->r + 1) - B->r, j % (2 * B->r + 1) - B->r};
    } else {
        int j = 1;
        offs[0] = {0, 0};
        for (int m = -B->r; m <= B->r; ++m) if (m) offs[j++] = {m, 0};
        for (int m = -B->r; m <= B->r; ++m) if (m) offs[j++] = {0, m};
    }
    std::vector<int> order(np);
    for (int j = 0; j < np; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return offs[a] < offs[b]; });
    long long tiles = 0;
    int maxp = 0;
    std::vector<int> passes(n);
    for (int g = 0; g < n; ++g) {
        BatchGrid<C> &G = hg[g];
        G.ny = (int)B->ny[g];
        G.nx = (int)B->nx[g];
        const int64_t T = B->T[g];
        G.passes = (int)((T + B->kb - 1) / B->kb);
        G.k_first = (int)(T - (int64_t)(G.passes - 1) * B->kb);
        G.bands = (G.nx + bw - 1) / bw;
        G.chunks = (G.ny + B->ly - 1) / B->ly;
        G.tile_base = (int)tiles;
        tiles += (long long)G.bands * G.chunks;
        for (int j = 0; j < np; ++j) G.w[j] = conv_w<C>(B->wts[(size_t)g * B->np + order[j]]);
        passes[g] = G.passes;
        maxp = std::max(maxp, G.passes);
    }
    B->ntiles = tiles;
    // dependency lists per band (columns) and per chunk (rows): the tiles of
    // the same grid whose output range meets the input window, wrapped for
    // periodic grids and clipped for Dirichlet ones
    const int hx = (32 * Traits<DT>::V - bw) / 2, hy = B->r * B->kb;
    std::vector<int> dep_off, dep_list;
    auto add_list = [&](int64_t lo, int64_t hi, int64_t n, int tile, int ntiles, bool periodic) {
        std::vector<char> hit(ntiles, 0);
        for (int64_t x = lo; x < hi; ++x) {
            int64_t xx = x;
            if (xx < 0 || xx >= n) {
                if (!periodic) continue;
                xx = ((xx % n) + n) % n;
            }
            hit[(int)(xx / tile < ntiles ? xx / tile : ntiles - 1)] = 1;
        }
        for (int t = 0; t < ntiles; ++t) if (hit[t]) dep_list.push_back(t);
        dep_off.push_back((int)dep_list.size());
    };
    const bool per = B->bkind == STENCIL_PERIODIC;
    for (int g = 0; g < n; ++g) {
        BatchGrid<C> &G = hg[g];
        G.boff = (int)dep_off.size();
        dep_off.push_back((int)dep_list.size());
        for (int b = 0; b < G.bands; ++b)
            add_list((int64_t)b * bw - hx, std::min<int64_t>((int64_t)(b + 1) * bw, G.nx) + hx, G.nx, bw, G.bands, per);
        G.coff = (int)dep_off.size();
        dep_off.push_back((int)dep_list.size());
        for (int c = 0; c < G.chunks; ++c)
            add_list((int64_t)c * B->ly - hy, std::min<int64_t>((int64_t)(c + 1) * B->ly, G.ny) + hy, G.ny, B->ly,
                     G.chunks, per);
    }
    std::vector<unsigned long long> items;
    for (int p = 0; p < maxp; ++p)
        for (int g = 0; g < n; ++g)
            if (p < passes[g])
                for (int t = 0; t < hg[g].bands * hg[g].chunks; ++t)
                    items.push_back((unsigned long long)g | ((unsigned long long)p << 16) |
                                    ((unsigned long long)t << 32));
    B->nitems = (long long)items.size();
    cudaError_t e = cudaMalloc(&B->d_grids, B->h_grids.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->d_items, sizeof(unsigned long long) * std::max<size_t>(1, items.size()));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_done, sizeof(int) * std::max<long long>(1, tiles));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_dep_off, sizeof(int) * dep_off.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->d_dep_list, sizeof(int) * std::max<size_t>(1, dep_list.size()));
    if (e != cudaSuccess) { cudaGetLastError(); set_error("batch allocation failed"); return STENCIL_ERR_OOM; }
    if (!items.empty())
        e = cudaMemcpy(B->d_items, items.data(), sizeof(unsigned long long) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(B->d_dep_off, dep_off.data(), sizeof(int) * dep_off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !dep_list.empty())
        e = cudaMemcpy(B->d_dep_list, dep_list.data(), sizeof(int) * dep_list.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { set_error("batch upload failed"); return STENCIL_ERR_CUDA; }
    if (B->ws.size() != (size_t)n) B->ws.assign(n, nullptr);
    for (int g = 0; g < n; ++g) {
        if (passes[g] < 2 || B->ws[g]) continue;   // a single pass reads `in` and writes `out` only
        e = cudaMalloc(&B->ws[g], B->bytes[g]);
        if (e != cudaSuccess) { cudaGetLastError(); set_error("batch workspace allocation failed"); return STENCIL_ERR_OOM; }
    }
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_kernel<DT, 1, STENCIL_BOX, 4>, BT_NW * 32, 0);
    B->grid_ctas = B->sm_count * std::max(1, bps);
    return STENCIL_OK;
}

template <int DT>
cudaError_t launch_batch(stencil_batch_s *B, cudaStream_t st) {
    using C = typename Traits<DT>::C;
    BatchParams<C> p;
    p.grids = static_cast<const BatchGrid<C> *>(B->d_grids);
    p.items = B->d_items;
    p.nitems = B->nitems;
    p.done = B->d_done;
    p.dep_off = B->d_dep_off;
    p.dep_list = B->d_dep_list;
    p.ctl = B->d_ctl;
    p.bkind = B->bkind;
    p.bval = conv_w<C>(B->bval);
    p.ly = B->ly;
    p.test_skip_publish = B->d_skip;
    const bool box = B->pattern == STENCIL_BOX;
    // the resident-worker bound keeps every dequeued item's dependencies running
    int bps = 0;
    auto pick = [&](auto k1, auto k2, auto k3, auto k4) { return B->kb == 1 ? k1 : B->kb == 2 ? k2 : B->kb == 3 ? k3 : k4; };
    auto kern = B->r == 1 ? (box ? pick(batch_kernel<DT, 1, STENCIL_BOX, 1>, batch_kernel<DT, 1, STENCIL_BOX, 2>,
                                        batch_kernel<DT, 1, STENCIL_BOX, 3>, batch_kernel<DT, 1, STENCIL_BOX, 4>)
                                 : pick(batch_kernel<DT, 1, STENCIL_STAR, 1>, batch_kernel<DT, 1, STENCIL_STAR, 2>,
                                        batch_kernel<DT, 1, STENCIL_STAR, 3>, batch_kernel<DT, 1, STENCIL_STAR, 4>))
                          : (box ? (B->kb == 1 ? batch_kernel<DT, 2, STENCIL_BOX, 1> : batch_kernel<DT, 2, STENCIL_BOX, 2>)
                                 : (B->kb == 1 ? batch_kernel<DT, 2, STENCIL_STAR, 1> : batch_kernel<DT, 2, STENCIL_STAR, 2>));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, BT_NW * 32, 0);
    const int ctas = B->sm_count * std::max(1, bps);
    kern<<<ctas, BT_NW * 32, 0, st>>>(p);
    return cudaGetLastError();
}

// free the schedule's device arrays and the captured graph (not the workspaces)
void release_schedule(stencil_batch_s *B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    cudaFree(B->d_grids);
    cudaFree(B->d_items);
    cudaFree(B->d_done);
    cudaFree(B->d_ctl);
    cudaFree(B->d_dep_off);
    cudaFree(B->d_dep_list);
    B->d_grids = nullptr;
    B->d_items = nullptr;
    B->d_done = nullptr;
    B->d_ctl = nullptr;
    B->d_dep_off = nullptr;
    B->d_dep_list = nullptr;
}

cudaError_t enqueue_batch(stencil_batch_s *B, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(B->d_done, 0, sizeof(int) * std::max<long long>(1, B->ntiles), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_ctl, 0, sizeof(BatchCtl), st);
    if (e != cudaSuccess) return e;
    switch (B->dtype) {
        case STENCIL_F32: return launch_batch<STENCIL_F32>(B, st);
        case STENCIL_I32: return launch_batch<STENCIL_I32>(B, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

extern "C" {

stencil_status_t stencil_batch_create(stencil_batch_t *out, int32_t n, int32_t dim, int32_t radius,
                                      const int64_t *shapes, const stencil_weights_t *weights, const int64_t *T,
                                      const stencil_boundary_t *boundary, int32_t dtype) {
    if (!out || !shapes || !weights || !T || !boundary || n < 1 || n > 65535) {
        set_error("invalid batch arguments");
        return STENCIL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (dim != 2) { set_error("batches support dim = 2"); return STENCIL_ERR_UNSUPPORTED; }
    if (radius < 1 || radius > 2) { set_error("batches support radius 1 or 2"); return STENCIL_ERR_UNSUPPORTED; }
    if (dtype != STENCIL_F32 && dtype != STENCIL_I32) { set_error("batches support F32 and I32"); return STENCIL_ERR_UNSUPPORTED; }
    if (boundary->kind != STENCIL_DIRICHLET && boundary->kind != STENCIL_PERIODIC) {
        set_error("invalid boundary kind");
        return STENCIL_ERR_INVALID_ARG;
    }
    const int pattern = weights[0].pattern;
    if (pattern != STENCIL_STAR && pattern != STENCIL_BOX) { set_error("invalid pattern"); return STENCIL_ERR_INVALID_ARG; }
    const int np = pattern == STENCIL_BOX ? (2 * radius + 1) * (2 * radius + 1) : 1 + 4 * radius;
    stencil_batch_s *B = new (std::nothrow) stencil_batch_s();
    if (!B) { set_error("host allocation failed"); return STENCIL_ERR_OOM; }
    B->n = n; B->r = radius; B->pattern = pattern; B->dtype = dtype; B->bkind = boundary->kind;
    B->bval = boundary->kind == STENCIL_DIRICHLET ? boundary->value : 0.0;
    B->kb = radius == 1 ? 4 : 2;
    for (int g = 0; g < n; ++g) {
        const int64_t ny = shapes[2 * g], nx = shapes[2 * g + 1];
        if (ny < 1 || nx < 1 || ny > (1 << 24) || nx > (1 << 24) || T[g] < 0 || T[g] > 65535 * (int64_t)B->kb ||
            weights[g].pattern != pattern || weights[g].count != np || !weights[g].w) {
            delete B;
            set_error("invalid shape, step count or weights for batch member " + std::to_string(g));
            return STENCIL_ERR_INVALID_ARG;
        }
        for (int j = 0; j < np; ++j) {
            const double w = weights[g].w[j];
            if (dtype == STENCIL_I32 && w != std::floor(w)) {
                delete B;
                set_error("integer mode needs integer weights");
                return STENCIL_ERR_INVALID_ARG;
            }
        }
        B->ny.push_back(ny);
        B->nx.push_back(nx);
        B->T.push_back(T[g]);
        for (int j = 0; j < np; ++j) B->wts.push_back(weights[g].w[j]);
        B->bytes.push_back((size_t)(ny * nx) * dtype_size(dtype));
    }
    cudaError_t e = cudaGetDevice(&B->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, B->device);
    if (e != cudaSuccess) { delete B; set_error("no CUDA device"); return STENCIL_ERR_CUDA; }
    B->np = np;
    stencil_status_t s = dtype == STENCIL_F32 ? build_batch<STENCIL_F32>(B) : build_batch<STENCIL_I32>(B);
    if (s != STENCIL_OK) { stencil_batch_destroy(B); return s; }
    *out = B;
    return STENCIL_OK;
}

stencil_status_t stencil_batch_destroy(stencil_batch_t B) {
    if (!B) return STENCIL_OK;
    cudaSetDevice(B->device);
    cudaDeviceSynchronize();
    release_schedule(B);
    cudaFree(B->d_skip);
    for (void *w : B->ws) cudaFree(w);
    delete B;
    return STENCIL_OK;
}

stencil_status_t stencil_batch_set_config(stencil_batch_t B, int32_t k, int32_t tile_rows) {
    if (!B || k < 0 || tile_rows < 0) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    const int kmax = B->r == 1 ? 4 : 2;
    const int kb = k == 0 ? kmax : k, ly = tile_rows == 0 ? BT_LY : tile_rows;
    if (kb > kmax || ly < 4 * B->r * kb || ly > (1 << 20)) {
        set_error("batch k must be 1.." + std::to_string(kmax) + " and tile rows at least 4 r k");
        return STENCIL_ERR_UNSUPPORTED;
    }
    for (int g = 0; g < B->n; ++g)
        if (B->T[g] > 65535 * (int64_t)kb) { set_error("a member's step count needs a larger k"); return STENCIL_ERR_UNSUPPORTED; }
    if (kb == B->kb && ly == B->ly) return STENCIL_OK;
    cudaDeviceSynchronize();
    release_schedule(B);
    B->kb = kb;
    B->ly = ly;
    B->last_in.clear();   // the grid table is uploaded again on the next run
    return B->dtype == STENCIL_F32 ? rebuild_batch<STENCIL_F32>(B) : rebuild_batch<STENCIL_I32>(B);
}

stencil_status_t stencil_batch_get_config(stencil_batch_t B, int32_t *k, int32_t *tile_rows) {
    if (!B || !k || !tile_rows) { set_error("null argument"); return STENCIL_ERR_INVALID_ARG; }
    *k = B->kb;
    *tile_rows = B->ly;
    return STENCIL_OK;
}

stencil_status_t stencil_batch_tune(stencil_batch_t B, const void *const *u_in, void *const *u_out, void *stream,
                                    double *best_ms) {
    if (!B || !u_in || !u_out) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int kmax = B->r == 1 ? 4 : 2;
    int bk = B->kb, bl = B->ly;
    float bms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    stencil_status_t s = STENCIL_OK;
    for (int k = 1; k <= kmax && s == STENCIL_OK; ++k)
        for (int ly : {32, 64, 128, 256}) {
            if (ly < 4 * B->r * k) continue;
            if (stencil_batch_set_config(B, k, ly) != STENCIL_OK) continue;
            s = stencil_batch_run(B, u_in, u_out, stream);   // warm-up (captures the graph)
            if (s != STENCIL_OK) break;
            float best = 1e30f;
            for (int rep = 0; rep < 3 && s == STENCIL_OK; ++rep) {
                cudaEventRecord(e0, st);
                s = stencil_batch_run(B, u_in, u_out, stream);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best = std::min(best, ms);
            }
            if (s == STENCIL_OK && best < bms) { bms = best; bk = k; bl = ly; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != STENCIL_OK) return s;
    s = stencil_batch_set_config(B, bk, bl);
    if (best_ms) *best_ms = bms;
    return s;
}

stencil_status_t stencil_batch_run(stencil_batch_t B, const void *const *u_in, void *const *u_out, void *stream) {
    if (!B || !u_in || !u_out) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    // every output must be disjoint from every input and from the other outputs
    struct Rng { const char *a; size_t n; int out; };
    std::vector<Rng> rs;
    for (int g = 0; g < B->n; ++g) {
        if (!u_in[g] || !u_out[g]) { set_error("null grid pointer"); return STENCIL_ERR_INVALID_ARG; }
        rs.push_back({static_cast<const char *>(u_in[g]), B->bytes[g], 0});
        rs.push_back({static_cast<const char *>(u_out[g]), B->bytes[g], 1});
    }
    std::sort(rs.begin(), rs.end(), [](const Rng &x, const Rng &y) { return x.a < y.a; });
    for (size_t i = 1; i < rs.size(); ++i)
        if (rs[i].a < rs[i - 1].a + rs[i - 1].n && (rs[i].out || rs[i - 1].out)) {
            set_error("batch outputs must not overlap inputs or other outputs");
            return STENCIL_ERR_INVALID_ARG;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // refresh the grid table when the caller's buffers change (stream-ordered,
    // before the graph); pageable source, so the host copy is taken at once
    bool changed = B->last_in.size() != (size_t)B->n;
    for (int g = 0; !changed && g < B->n; ++g) changed = B->last_in[g] != u_in[g] || B->last_out[g] != u_out[g];
    if (changed) {
        const size_t ds = B->grid_desc_size;
        for (int g = 0; g < B->n; ++g) {
            unsigned char *d = B->h_grids.data() + ds * g;
            const void *in = u_in[g];
            void *outp = u_out[g];
            memcpy(d, &in, sizeof(void *));
            memcpy(d + sizeof(void *), &outp, sizeof(void *));
            memcpy(d + 2 * sizeof(void *), &B->ws[g], sizeof(void *));
        }
        cudaError_t e = cudaMemcpyAsync(B->d_grids, B->h_grids.data(), B->h_grids.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { set_error(std::string("grid table upload: ") + cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
        B->last_in.assign(u_in, u_in + B->n);
        B->last_out.assign(u_out, u_out + B->n);
    }
    if (!B->exec) {
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) { set_error("stream creation failed"); return STENCIL_ERR_CUDA; }
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = enqueue_batch(B, cs);
            e = cudaStreamEndCapture(cs, &B->graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            set_error(std::string("graph capture: ") + cudaGetErrorString(e));
            return STENCIL_ERR_CUDA;
        }
    }
    for (int g = 0; g < B->n; ++g)   // members with T = 0 are copied
        if (B->T[g] == 0) {
            cudaError_t ce = cudaMemcpyAsync(u_out[g], u_in[g], B->bytes[g], cudaMemcpyDeviceToDevice, st);
            if (ce != cudaSuccess) { set_error(cudaGetErrorString(ce)); return STENCIL_ERR_CUDA; }
        }
    cudaError_t e = cudaGraphLaunch(B->exec, st);
    if (e != cudaSuccess) { set_error(std::string("graph launch: ") + cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
    return STENCIL_OK;
}

stencil_status_t stencil_batch_get_device_status(stencil_batch_t B) {
    if (!B) { set_error("null batch"); return STENCIL_ERR_INVALID_ARG; }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
    BatchCtl h;
    e = cudaMemcpy(&h, B->d_ctl, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return STENCIL_ERR_CUDA; }
    if (h.status) { set_error("a batch dependency wait gave up"); return (stencil_status_t)h.status; }
    return STENCIL_OK;
}

stencil_status_t stencil_batch_launch_count(stencil_batch_t B, int64_t *launches) {
    if (!B || !launches) { set_error("invalid argument"); return STENCIL_ERR_INVALID_ARG; }
    *launches = 1;
    return STENCIL_OK;
}

// Test hook (not in the public header): makes item `q` skip its completion
// publish, so that the items depending on it must give up their bounded
// waits -- host-side fault injection for the timeout path.  q < 0 disables.
stencil_status_t stencil_batch_test_skip_publish(stencil_batch_t B, int64_t q) {
    if (!B) return STENCIL_ERR_INVALID_ARG;
    if (!B->d_skip) {
        if (cudaMalloc(&B->d_skip, sizeof(int)) != cudaSuccess) return STENCIL_ERR_OOM;
    }
    int v = (int)q;
    if (cudaMemcpy(B->d_skip, &v, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return STENCIL_ERR_CUDA;
    // the captured graph holds the old parameters: capture again
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    return STENCIL_OK;
}

}  // extern "C"
