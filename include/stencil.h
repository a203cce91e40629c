/*
 * stencil.h -- C ABI of the GB300 (sm_103a) iterated-stencil library.
 *
 * The library advances d-dimensional grids (d = 1, 2, 3) by T Jacobi time
 * steps of a star or box stencil of order r.  The operation is the one the
 * paper defines in Section 1: every grid point at time t+1 is a weighted sum
 * of its (2r+1)-per-dimension neighbours at time t, the time loop outermost.
 * Several time steps are fused into each pass over HBM, the GPU counterpart
 * of the paper's time-loop unroll-and-jam (Section 3.3, Algorithm 1).
 *
 * Conventions (the paper leaves them open; the library fixes them):
 *   grid     interior points only, dense, row-major, outermost dimension
 *            first, innermost (unit-stride, "x") dimension last;
 *   update   u_{t+1}[x] = sum_{o in S} w_o * u_t(x + o)   (a correlation);
 *   S        box: [-r, r]^d;  star: {0} and {+-j e_a : 1 <= j <= r};
 *   weights  compact order.  box: (2r+1)^d values, offsets lexicographic
 *            (o_0, ..., o_{d-1}) with the innermost dimension fastest;
 *            star: 1 + 2dr values [centre, axis 0: -r..-1, +1..+r, axis 1:
 *            ..., ...], axis 0 being the outermost dimension;
 *   boundary DIRICHLET: out-of-domain values are the constant `value` at
 *            every time level; PERIODIC: indices wrap modulo the extent;
 *   order    each sum is evaluated as one multiply followed by fused
 *            multiply-adds over the offsets in lexicographic order, so every
 *            fusion depth k gives bit-identical results;
 *   dtypes   F64 (FP64 math), F32 (FP32 math), BF16 and F16 (storage only:
 *            FP32 math, one round-to-nearest-even per fused pass), I32
 *            (uint32 wraparound arithmetic, bit-exact; weights and the
 *            boundary value must be integers).
 *
 * Ownership and errors (all entry points):
 *   - Device pointers are plain CUDA device addresses (for example a torch
 *     tensor's data_ptr()), owned by the caller, contiguous, of the plan's
 *     dtype and shape.  `stream` is a cudaStream_t (NULL = legacy default).
 *   - All device work is enqueued asynchronously on `stream`; host pointers
 *     are only read during the call unless stated otherwise.
 *   - Argument, shape and support errors are returned before anything is
 *     enqueued.  CUDA errors return STENCIL_ERR_CUDA.  A device-side bounded
 *     wait that gives up records STENCIL_ERR_TIMEOUT in the plan's device
 *     status word, read by stencil_get_device_status.
 *   - No C++ exception crosses this interface.  A plan may be used by one
 *     host thread at a time; calls on different streams with the same plan
 *     share its workspace and must not overlap.
 *   - stencil_last_error() returns a message for the calling thread's most
 *     recent failing call.
 */
#ifndef STENCIL_GB300_H
#define STENCIL_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stencil_plan_s *stencil_plan_t;
typedef struct stencil_batch_s *stencil_batch_t;

typedef enum {
    STENCIL_OK = 0,
    STENCIL_ERR_INVALID_ARG = 1,
    STENCIL_ERR_UNSUPPORTED = 2,
    STENCIL_ERR_OOM = 3,
    STENCIL_ERR_CUDA = 4,
    STENCIL_ERR_TIMEOUT = 5,
    STENCIL_ERR_INTERNAL = 6
} stencil_status_t;

typedef enum { STENCIL_F64 = 0, STENCIL_F32 = 1, STENCIL_BF16 = 2, STENCIL_F16 = 3, STENCIL_I32 = 4 } stencil_dtype_t;
typedef enum { STENCIL_STAR = 0, STENCIL_BOX = 1 } stencil_pattern_t;
typedef enum { STENCIL_DIRICHLET = 0, STENCIL_PERIODIC = 1 } stencil_boundary_kind_t;

/* Which kernels stencil_run uses.  FUSED: k steps per pass (the default);
 * the passes of exactly k steps run as one persistent launch whose tiles
 * wait on their neighbours' completion of the previous pass.
 * PLAIN: one step per launch, each thread reading its own neighbours -- the
 * one-step-per-launch sweep the fused path is measured against.
 * FUSED_PER_PASS: the fused kernels with one launch per pass.
 * TESSELLATE: the paper's tessellate tiling (Section 3.4): time tiles of h
 * levels (h = the plan's k, default 8; any h with 2 h r no longer than a
 * segment), each in d + 1 stages of concurrent shrinking / expanding tiles
 * that together update every point once per level -- no redundant work, one
 * launch per stage; segments of the plan's tile length (default 2048, 64, 16
 * points in 1D, 2D, 3D, at least 2 h r; a tile must stay below 2^31 points).  Results are
 * bit-identical to the other forms.  On GB300 it runs well below the fused
 * forms (each stage is a launch, each level a CTA barrier, and a tile loads and
 * writes back both level buffers): it is there as the paper's scheme, not as a
 * fast path. */
typedef enum {
    STENCIL_VARIANT_FUSED = 0,
    STENCIL_VARIANT_PLAIN = 1,
    STENCIL_VARIANT_FUSED_PER_PASS = 2,
    STENCIL_VARIANT_TESSELLATE = 3
} stencil_variant_t;

/* Stencil coefficients: `count` values in compact order (see above). */
typedef struct {
    int32_t pattern; /* stencil_pattern_t */
    int32_t count;   /* must equal (2r+1)^d (box) or 1+2dr (star) */
    const double *w; /* host pointer, read during the call */
} stencil_weights_t;

typedef struct {
    int32_t kind;    /* stencil_boundary_kind_t */
    double value;    /* Dirichlet value (ignored when periodic) */
} stencil_boundary_t;

/* ------------------------------------------------------------------ plans */

/* Create a plan for one grid geometry (Section 1: dimension d, order r,
 * weighted sum over the neighbourhood).  `shape` holds d extents, outermost
 * first, each >= 1.  1 <= dim <= 3, 1 <= radius <= 3.  Allocates nothing on
 * the device until first use.  On success *out owns the plan. */
stencil_status_t stencil_plan_create(stencil_plan_t *out, int32_t dim, int32_t radius, const int64_t *shape,
                                     const stencil_weights_t *weights, const stencil_boundary_t *boundary,
                                     int32_t dtype);

/* Release a plan and its device workspace (synchronises its device). */
stencil_status_t stencil_plan_destroy(stencil_plan_t plan);

/* Fusion depth k (time steps per pass, the paper's unrolling factor of
 * Section 3.3).  0 selects the plan's default; values above the kernels'
 * limit for this geometry return STENCIL_ERR_UNSUPPORTED. */
stencil_status_t stencil_plan_set_k(stencil_plan_t plan, int32_t k);
stencil_status_t stencil_plan_get_k(stencil_plan_t plan, int32_t *k);
/* Largest k the fused kernels accept for this plan. */
stencil_status_t stencil_plan_max_k(stencil_plan_t plan, int32_t *kmax);

/* Select FUSED (default), PLAIN or FUSED_PER_PASS kernels for stencil_run;
 * get returns the kernels stencil_run uses now (after stencil_plan_tune, the
 * tuner's choice). */
stencil_status_t stencil_plan_set_variant(stencil_plan_t plan, int32_t variant);
stencil_status_t stencil_plan_get_variant(stencil_plan_t plan, int32_t *variant);

/* Tile length of the fused kernels along the outermost dimension: in 2D the
 * rows one warp job advances (at least max(4 r k, 16)), in 3D the z planes
 * one CTA job advances (at least max(4 r k, 8)), in 1D the vector sets of
 * 32 x (2 FP64, else 4) elements one warp job of the persistent launch
 * advances; at most the grid's extent is used.  0 selects
 * the default (about two to three jobs per resident warp or CTA per pass). */
stencil_status_t stencil_plan_set_tile_rows(stencil_plan_t plan, int32_t rows);
stencil_status_t stencil_plan_get_tile_rows(stencil_plan_t plan, int32_t *rows);

/* Warps per CTA of the 2D fused kernels (each warp streams its own jobs; the
 * block size sets how many share an SM's scheduling slot and shared-memory
 * carve-out): 1..8, 0 = the default of 4.  The 1D and 3D kernels have fixed
 * block sizes (a 3D CTA's 16 warps make up its 64-row window). */
stencil_status_t stencil_plan_set_block_warps(stencil_plan_t plan, int32_t warps);
stencil_status_t stencil_plan_get_block_warps(stencil_plan_t plan, int32_t *warps);

/* Autotune the fusion depth, the launch form and the tile length:
 * times stencil_run for the one-step kernel and, for every supported k, the
 * fused kernels with one launch per pass and the persistent multi-pass
 * launch with each of a few tile lengths, on
 * plan-owned buffers holding zeros, with CUDA events on `stream`, and keeps
 * the fastest (for tiny or FP64-pipe-bound grids the one-step kernel can
 * win).  Synchronises `stream`.  `T` is the step count to tune for; best_k
 * (may be NULL) receives the chosen k, or 0 when the one-step kernel won;
 * best_ms (may be NULL) its time; the chosen launch form and tile length are
 * read with stencil_plan_get_variant and stencil_plan_get_tile_rows.
 * stencil_plan_set_k and stencil_plan_set_variant discard the choice of
 * kernel. */
stencil_status_t stencil_plan_tune(stencil_plan_t plan, int64_t T, void *stream, int32_t *best_k, double *best_ms);

/* Number of kernel launches stencil_run makes for T steps with the current
 * variant and k: T plain steps, ceil(T/k) fused passes, or for the
 * persistent form one launch plus one for a last pass of T mod k steps. */
stencil_status_t stencil_plan_launch_count(stencil_plan_t plan, int64_t T, int64_t *launches);

/* Short text naming the kernel, k and tiling the plan uses (for logs). */
stencil_status_t stencil_plan_describe(stencil_plan_t plan, char *buf, int32_t len);

/* ------------------------------------------------------------------ sweep */

/* u_out := T Jacobi steps applied to u_in (Section 1; fused per Section 3.3).
 * Both are device pointers of the plan's shape and dtype; u_in is only read;
 * u_out must not overlap u_in.  T = 0 copies.  Intermediate passes use a
 * plan-owned device buffer of one grid; the persistent launch also keeps a
 * small block of per-tile counters.  Both are allocated on first use (and the
 * counters regrown when a new k or tile length needs more), so a call that is
 * to be captured into a CUDA graph should follow one uncaptured call with the
 * same settings.  Asynchronous on `stream`; a device-side timeout is read
 * with stencil_get_device_status.  Plans are not safe for concurrent use on
 * several streams. */
stencil_status_t stencil_run(stencil_plan_t plan, const void *u_in, void *u_out, int64_t T, void *stream);

/* Same computation on HOST buffers: copies h_in to the device, runs T steps,
 * copies the result to h_out, and synchronises `stream` before returning.
 * Uses two plan-owned device grids.  Pinned host memory makes the copies
 * asynchronous engine transfers; pageable memory works but is slower. */
stencil_status_t stencil_run_host(stencil_plan_t plan, const void *h_in, void *h_out, int64_t T, void *stream);

/* In-place sweep (2D plans): u := T steps applied to u, with one grid of
 * memory instead of two -- the GPU form of the paper's in-place update
 * (Section 3.3, last paragraph: with k = 2 the input and output of a pass sit
 * at even time levels, so one array suffices).  Tiles advance k steps per pass
 * as in stencil_run (k = the plan's k, at most 4 for r = 1, 2 for r = 2 and 1
 * for r = 3; the update order and so the
 * result are stencil_run's, bit for bit) and overwrite their own cells; the
 * cells within r k rows or H >= r k columns of every tile's border, which
 * neighbouring tiles read, are kept in two plan-owned ring buffers (the pass
 * before's values and this pass's), about 2 (2 r k / Ly + 2 H / BW) of a
 * grid.  One launch per pass plus one to fill the rings.  u is a device
 * pointer of the plan's shape and dtype. */
stencil_status_t stencil_run_inplace(stencil_plan_t plan, void *u, int64_t T, void *stream);
/* Device bytes stencil_run_inplace uses beyond the grid itself (the two ring
 * buffers), for the plan's current k; stencil_run uses one grid. */
stencil_status_t stencil_inplace_workspace_bytes(stencil_plan_t plan, int64_t *bytes);

/* Variable-coefficient sweep: u_out := T steps of
 *     u_{t+1}[x] = sum_o c_o[x] * u_t(x + o)
 * with a coefficient per offset and per grid point (the Section 1 sweep with
 * its weights made fields; not in the paper).  The plan gives the geometry,
 * pattern, radius, boundary and dtype (F32, F64 or I32); its weights are not
 * used.  `coef` is a device array of np x N values of the arithmetic type
 * (float for F32, double for F64, int32 for I32), offset-major in compact
 * order: coef[j * N + x] multiplies the j-th compact offset at point x.
 * Terms are summed in the same order as stencil_run, so a constant field
 * reproduces it bit for bit.  2D plans fuse k steps per pass (the plan's k,
 * at most 4 for r = 1 and 2 for r = 2: the coefficient planes are read once
 * per pass, (2 + np) s bytes per point and pass); r = 3 and 1D/3D plans run
 * one step per launch.  u_out must not overlap u_in; a plan-owned grid holds
 * the intermediate passes. */
stencil_status_t stencil_run_vc(stencil_plan_t plan, const void *coef, const void *u_in, void *u_out, int64_t T,
                                void *stream);

/* Reverse-mode derivative of stencil_run_vc (not in the paper: neither the
 * coefficient fields nor the derivative are).  For lam_T = grad_uT = dL/du_T
 * of a loss L of u_T = T steps applied to u0 with coefficient field `coef`:
 *     grad_coef[o][x] = dL/dc_o[x] = sum_t lam_{t+1}[x] * u_t(x + o)
 *                       (the boundary value where x + o lies outside a Dirichlet domain)
 *     lam_t[y]        = sum_o c_o[y - o] * lam_{t+1}[y - o]
 *                       (y - o wrapped on periodic axes, dropped outside a Dirichlet domain)
 *     grad_u0         = lam_0.
 * F32 and F64 plans, d = 1..3.  coef and grad_coef: np x N values in the
 * plan's arithmetic type, compact offset order (stencil_run_vc's layout);
 * grad_coef is overwritten.  The forward states come from checkpoints every
 * ckpt_every steps (1..T) taken by a forward sweep inside the call, each
 * segment's inner states recomputed one step at a time; the workspace
 * (ceil(T / ckpt_every) + ckpt_every grids) is plan-owned.  grad_uT, grad_u0,
 * u0 must not overlap each other or coef.  Enqueued on `stream`. */
stencil_status_t stencil_adjoint_vc(stencil_plan_t plan, const void *coef, const void *u0, const void *grad_uT,
                                    int64_t T, int32_t ckpt_every, void *grad_u0, void *grad_coef, void *stream);

/* Many host grids in a row, pipelined: h_out[i] := T steps applied to
 * h_in[i] for i < n (host buffers of the plan's shape and dtype, each read or
 * written during the call).  Two input and two output grids are kept on the
 * device so that the host-to-device copy of grid i + 1 and the
 * device-to-host copy of grid i - 1 run on two copy streams while grid i is
 * swept on `stream`: with pinned buffers the time per grid approaches the
 * longest of the three instead of their sum.  Synchronises `stream` before
 * returning. */
stencil_status_t stencil_run_host_many(stencil_plan_t plan, int64_t n, const void *const *h_in, void *const *h_out,
                                       int64_t T, void *stream);

/* ---------------------------------------------------------------- batches */

/* The paper has no batched form: its experiments advance one grid at a time
 * (Section 4).  This entry point serves the batched workload of this
 * library's specification (256 periodic 2D 9-point grids of uneven sizes and
 * step counts in one persistent, graph-captured launch); each member's result
 * is the Section 1 sweep of that member. */

/* A batch of `n` independent 2D grids of one dtype, order and boundary, each
 * with its own shape (shapes: n x dim, outermost first), coefficients
 * (weights[i]) and step count (T[i] >= 0).  All grids are advanced together
 * by one persistent kernel that takes (pass, grid, tile) work items from a
 * queue, waiting with bounded spins for the neighbouring tiles of the
 * previous pass; the first stencil_batch_run captures that launch into a
 * CUDA graph which later calls replay.  The batch owns one workspace grid per
 * member.  Only dim = 2 and dtype F32 / I32 are supported. */
stencil_status_t stencil_batch_create(stencil_batch_t *out, int32_t n, int32_t dim, int32_t radius,
                                      const int64_t *shapes, const stencil_weights_t *weights, const int64_t *T,
                                      const stencil_boundary_t *boundary, int32_t dtype);
stencil_status_t stencil_batch_destroy(stencil_batch_t batch);

/* u_out[i] := T[i] steps applied to u_in[i] for every member.  u_in, u_out:
 * host arrays of n device pointers (read during the call).  Every u_out[i]
 * must differ from every u_in[j].  Bounded waits that give up record
 * STENCIL_ERR_TIMEOUT, read by stencil_batch_get_device_status. */
stencil_status_t stencil_batch_run(stencil_batch_t batch, const void *const *u_in, void *const *u_out,
                                   void *stream);
stencil_status_t stencil_batch_get_device_status(stencil_batch_t batch);
/* The batch's fusion depth k (1..4 for r = 1, 1..2 for r = 2; 0 = the
 * largest) and tile height in rows (at least 4 r k; 0 = 64): every member's
 * passes advance k steps (the first the remainder of T), in tiles of one
 * 120-column band x tile_rows rows.  Changing them rebuilds the schedule and
 * recaptures the graph on the next run. */
stencil_status_t stencil_batch_set_config(stencil_batch_t batch, int32_t k, int32_t tile_rows);
stencil_status_t stencil_batch_get_config(stencil_batch_t batch, int32_t *k, int32_t *tile_rows);
/* Autotune k and the tile height on the caller's buffers (the batch is run
 * several times per candidate, timed with CUDA events on `stream`) and keep
 * the fastest; best_ms (may be NULL) receives its time. */
stencil_status_t stencil_batch_tune(stencil_batch_t batch, const void *const *u_in, void *const *u_out, void *stream,
                                    double *best_ms);
/* Kernel launches per stencil_batch_run (the graph's kernel nodes). */
stencil_status_t stencil_batch_launch_count(stencil_batch_t batch, int64_t *launches);

/* ----------------------------------------------------------------- adjoint */

/* The paper does not differentiate the sweep.  This entry point serves the
 * differentiation workload of this library's specification (gradients of a
 * loss of u_T with respect to u_0 and the weights, recomputed from
 * checkpoints); the forward map it differentiates is the Section 1 sweep. */

/* Reverse-mode derivative of u_T = (T steps)(u0) for F32 plans: given
 * grad_uT = dL/du_T (device, plan shape), writes grad_u0 = dL/du0 (device,
 * plan shape) and grad_w[j] = dL/dw_j (device, `count` doubles, compact
 * order).  The transposed sweep runs backward in time; forward states are
 * recomputed from checkpoints stored every `ckpt_every` steps (1 <= ckpt_every
 * <= T): this call first runs stencil_run_checkpointed into plan-owned
 * checkpoints, then stencil_adjoint_from_checkpoints (the plan keeps
 * ceil(T/ckpt_every) + ckpt_every + 1 grids of workspace).
 * With a Dirichlet boundary the weight gradient includes the boundary value's
 * contributions. */
stencil_status_t stencil_adjoint_run(stencil_plan_t plan, const void *u0, const void *grad_uT, int64_t T,
                                     int32_t ckpt_every, void *grad_u0, double *grad_w, void *stream);

/* The forward sweep of an F32 plan with checkpoints kept for the adjoint:
 * u_T := T steps of u0 (as stencil_run, in segments of ckpt_every steps) and
 * ckpts[m] := the state after (m + 1) ckpt_every steps for
 * m = 0 .. ceil(T / ckpt_every) - 2 (caller-owned device buffer of that many
 * grids; may be NULL when T <= ckpt_every).  The checkpoints cost no extra
 * sweep: each segment writes its result there directly. */
stencil_status_t stencil_run_checkpointed(stencil_plan_t plan, const void *u0, void *u_T, int64_t T,
                                          int32_t ckpt_every, void *ckpts, void *stream);
/* The backward sweep of stencil_adjoint_run from checkpoints that
 * stencil_run_checkpointed took (same u0, T and ckpt_every): grad_u0 and
 * grad_w as there, without re-running the forward sweep.  The weight gradient
 * sums each thread's products of one step in FP32 and everything above that
 * (warps, blocks, steps) in FP64. */
stencil_status_t stencil_adjoint_from_checkpoints(stencil_plan_t plan, const void *u0, const void *ckpts,
                                                  const void *grad_uT, int64_t T, int32_t ckpt_every, void *grad_u0,
                                                  double *grad_w, void *stream);

/* -------------------------------------------------------------- reductions */

/* Not in the paper: the FP64 conservation and norm reductions of this
 * library's specification (mass, squared norm, the adjoint workload's loss). */

typedef enum {
    STENCIL_REDUCE_SUM = 0,       /* sum u                       */
    STENCIL_REDUCE_SUMSQ = 1,     /* sum u^2                     */
    STENCIL_REDUCE_HALF_SQDIST = 2 /* 0.5 * sum (u - target)^2  */
} stencil_reduce_op_t;

/* FP64 reduction over n elements of dtype `dtype` (F64, F32, BF16, F16):
 * elements are widened to FP64 and summed in a fixed order (deterministic).
 * `target` is used only by HALF_SQDIST.  The result is written to the device
 * double *out.  Per-block partial sums live in a library-owned device buffer
 * of the current device, allocated on first use and grown as needed. */
stencil_status_t stencil_reduce(int32_t dtype, int64_t n, const void *u, const void *target, int32_t op,
                                double *out, void *stream);

/* Allocation-free form of stencil_reduce, for callers that cannot allocate
 * device memory when they reduce: devices or drivers without stream-ordered
 * memory pools (stencil_reduce takes its partial-sum buffer with
 * cudaMallocAsync), applications whose caching allocator already holds nearly
 * all free device memory, and latency-critical loops that must not enter an
 * allocator.  Same arguments, same partition and summation order and so a
 * bit-identical result to stencil_reduce, but the per-block partial sums live
 * in a library-static device array of 1024 doubles (8 KiB), which every GPU
 * that loads the library holds until the process exits; no cudaMalloc,
 * cudaMallocAsync, cudaFree or other allocating call is made.  The reduction
 * never uses more than 1024 partial sums, so n is not limited by the array.
 * The first call on a device (and the first after that device's context was
 * re-created, e.g. by cudaDeviceReset) looks up the array's device address
 * with cudaGetSymbolAddress, with that device current, and caches it; make
 * that first call before any stream capture.  Every call reuses the same
 * array (each call writes every partial it reads, so nothing needs clearing):
 * calls whose kernels overlap on the GPU -- on different streams without
 * ordering between them -- race and can return wrong sums.
 * The paper has no counterpart to this entry point. */
stencil_status_t stencil_reduce_noalloc(int32_t dtype, int64_t n, const void *u, const void *target, int32_t op,
                                        double *out, void *stream);

/* -------------------------------------------------------------- diagnostics */

/* Measured fused multiply-add throughput of the current device for `dtype`
 * (F32 or F64), in FMAs per second: independent FMA chains on every SM, timed
 * with CUDA events on `stream` (synchronises it).  Not in the paper: it gives
 * the compute roof against which the sweeps that are bound by the FP32 pipe
 * (the 3D 27-point box) or the FP64 pipe (every FP64 sweep on this GPU) are
 * graded, the way a copy kernel gives the HBM roof. */
stencil_status_t stencil_probe_fma_rate(int32_t dtype, double *fma_per_s, void *stream);

/* Host-only (no device needed): the level counts of the tessellate tiling
 * that STENCIL_VARIANT_TESSELLATE uses for a grid of `shape` (dim extents),
 * radius, `levels` per time tile, segment length `tile` and periodic (1) or
 * Dirichlet (0) boundary.  counts[(dim + 1) x N] receives, for each stage s
 * and point x, the number of levels at which stage s updates x: in 1D stage 0
 * gives each segment the paper's (0, 1, .., h, .., 1, 0) profile, stage 1 the
 * complement, and the stages sum to `levels` at every point (Section 3.4,
 * Fig. 6).  STENCIL_ERR_INVALID_ARG when a segment is shorter than
 * 2 levels radius or the grid has more than 2^26 points. */
stencil_status_t stencil_tess_counts(int32_t dim, const int64_t *shape, int32_t radius, int32_t levels, int32_t tile,
                                     int32_t periodic, int32_t *counts);

/* ------------------------------------------------------------------ status */

/* Synchronises the plan's device and returns (then clears) its device
 * status word: STENCIL_OK or STENCIL_ERR_TIMEOUT. */
stencil_status_t stencil_get_device_status(stencil_plan_t plan);
const char *stencil_status_string(stencil_status_t status);
const char *stencil_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_GB300_H */
