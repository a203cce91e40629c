/*
 * oracle.c -- FP64 / uint32 reference of the iterated Jacobi stencil sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU library computes.  Only tests/, the smoke
 * check and bench.py's CPU-baseline leg may call it.  It shares no code,
 * header, table or helper with the CUDA path, and includes nothing from it.
 *
 * Definition followed (paper, Section 1): a d-dimensional stencil of order r
 * updates every grid point iteratively along the time dimension; the value of
 * a point at time t+1 is a weighted sum of (2r+1) points per dimension at time
 * t; the naive code is d+1 nested loops with time outermost.  The method's
 * time-loop unroll-and-jam (Section 3.3, Algorithm 1) and tessellate tiling
 * (Section 3.4) only reorder independent point updates and keep Jacobi
 * semantics (old values are preserved in "vrl"), so their result is exactly
 * this loop nest.
 *
 * Readings fixed here (the paper is silent on them):
 *   - update is a correlation: u_{t+1}[x] = sum_o w_o * u_t(x + o);
 *   - box pattern: o in [-r, r]^d; star pattern: o = 0 or o = +-j e_a,
 *     1 <= j <= r (the paper's 2D9P and 3D27P are box, the other four star);
 *   - compact weight order: box lexicographic over (o_0..o_{d-1}), innermost
 *     (last, unit-stride) dimension fastest; star [centre, axis 0: -r..-1,
 *     +1..+r, axis 1: ..., ...];
 *   - out-of-domain values: Dirichlet -> the constant bval at every t;
 *     periodic -> index taken modulo the extent;
 *   - each sum is accumulated in FP64 over the offsets in lexicographic
 *     order, starting from 0, without contraction (-ffp-contract=off);
 *   - integer mode computes the same sums in uint32 wraparound arithmetic.
 *
 * Every entry point returns 0 on success, -1 on an invalid argument and -2
 * when memory runs out.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXPTS 343 /* box, d = 3, r = 3 */

typedef struct {
    int d, r, pattern, np;
    int64_t n[3];          /* padded to 3 dims, leading extents 1 */
    int off[OR_MAXPTS][3]; /* padded offsets, evaluation (lexicographic) order */
    int cidx[OR_MAXPTS];   /* compact index of the j-th evaluated offset */
    int bkind;
} or_geom;

int oracle_npoints(int d, int r, int pattern)
{
    if (d < 1 || d > 3 || r < 1 || r > 3) return -1;
    if (pattern == 1) { int p = 1; for (int a = 0; a < d; ++a) p *= 2 * r + 1; return p; }
    if (pattern == 0) return 1 + 2 * d * r;
    return -1;
}

/* Offsets in compact weight order, np x d ints (outermost dimension first). */
int oracle_offsets(int d, int r, int pattern, int32_t *off)
{
    int np = oracle_npoints(d, r, pattern);
    if (np < 0 || !off) return -1;
    if (pattern == 1) {
        for (int j = 0; j < np; ++j) {
            int rem = j;
            for (int a = d - 1; a >= 0; --a) { off[j * d + a] = rem % (2 * r + 1) - r; rem /= 2 * r + 1; }
        }
    } else {
        int j = 0;
        for (int a = 0; a < d; ++a) off[a] = 0;
        j = 1;
        for (int a = 0; a < d; ++a) {
            for (int m = -r; m <= r; ++m) {
                if (m == 0) continue;
                for (int b = 0; b < d; ++b) off[j * d + b] = (b == a) ? m : 0;
                ++j;
            }
        }
    }
    return np;
}

static int lex_less(const int *a, const int *b)
{
    for (int i = 0; i < 3; ++i) { if (a[i] != b[i]) return a[i] < b[i]; }
    return 0;
}

static int or_setup(or_geom *g, int d, int r, int pattern, const int64_t *n, int bkind)
{
    int32_t raw[OR_MAXPTS * 3];
    if (!n || (bkind != 0 && bkind != 1)) return -1;
    int np = oracle_offsets(d, r, pattern, raw);
    if (np < 0) return -1;
    g->d = d; g->r = r; g->pattern = pattern; g->np = np; g->bkind = bkind;
    for (int a = 0; a < 3; ++a) g->n[a] = 1;
    for (int a = 0; a < d; ++a) { if (n[a] < 1) return -1; g->n[3 - d + a] = n[a]; }
    for (int j = 0; j < np; ++j) {
        g->cidx[j] = j;
        for (int a = 0; a < 3; ++a) g->off[j][a] = 0;
        for (int a = 0; a < d; ++a) g->off[j][3 - d + a] = raw[j * d + a];
    }
    /* insertion sort into lexicographic order (o_0, ..., o_{d-1}) */
    for (int i = 1; i < np; ++i) {
        int to[3] = { g->off[i][0], g->off[i][1], g->off[i][2] }, tc = g->cidx[i];
        int k = i - 1;
        while (k >= 0 && lex_less(to, g->off[k])) {
            for (int a = 0; a < 3; ++a) g->off[k + 1][a] = g->off[k][a];
            g->cidx[k + 1] = g->cidx[k];
            --k;
        }
        for (int a = 0; a < 3; ++a) g->off[k + 1][a] = to[a];
        g->cidx[k + 1] = tc;
    }
    return 0;
}

static int64_t wrap(int64_t i, int64_t n) { int64_t m = i % n; return m < 0 ? m + n : m; }

/* 1 and the linear index if (i0,i1,i2) resolves to a stored value, 0 if it is
 * a Dirichlet boundary cell. */
static int resolve(const or_geom *g, int64_t i0, int64_t i1, int64_t i2, int64_t *lin)
{
    int64_t c[3] = { i0, i1, i2 };
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= g->n[a]) {
            if (g->bkind == 0) return 0;
            c[a] = wrap(c[a], g->n[a]);
        }
    }
    *lin = (c[0] * g->n[1] + c[1]) * g->n[2] + c[2];
    return 1;
}

/* ---------------------------------------------------------------- forward */

static void step_f64(const or_geom *g, const double *w, double bval, const double *src, double *dst)
{
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    int64_t rows = n0 * n1;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t i0 = row / n1, i1 = row % n1;
        for (int64_t i2 = 0; i2 < n2; ++i2) {
            double acc = 0.0;
            for (int j = 0; j < g->np; ++j) {
                int64_t lin;
                double v = resolve(g, i0 + g->off[j][0], i1 + g->off[j][1], i2 + g->off[j][2], &lin) ? src[lin] : bval;
                acc = acc + w[g->cidx[j]] * v;
            }
            dst[(i0 * n1 + i1) * n2 + i2] = acc;
        }
    }
}

int oracle_run_f64(int d, int r, int pattern, const int64_t *n, const double *w, int bkind, double bval,
                   const double *u0, int64_t T, double *uT)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !w || !u0 || !uT || T < 0) return -1;
    int64_t N = g.n[0] * g.n[1] * g.n[2];
    double *a = (double *)malloc(sizeof(double) * N), *b = (double *)malloc(sizeof(double) * N);
    if (!a || !b) { free(a); free(b); return -2; }
    memcpy(a, u0, sizeof(double) * N);
    for (int64_t t = 0; t < T; ++t) { step_f64(&g, w, bval, a, b); double *s = a; a = b; b = s; }
    memcpy(uT, a, sizeof(double) * N);
    free(a); free(b);
    return 0;
}

static void step_u32(const or_geom *g, const uint32_t *w, uint32_t bval, const uint32_t *src, uint32_t *dst)
{
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    int64_t rows = n0 * n1;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t i0 = row / n1, i1 = row % n1;
        for (int64_t i2 = 0; i2 < n2; ++i2) {
            uint32_t acc = 0u;
            for (int j = 0; j < g->np; ++j) {
                int64_t lin;
                uint32_t v = resolve(g, i0 + g->off[j][0], i1 + g->off[j][1], i2 + g->off[j][2], &lin) ? src[lin] : bval;
                acc = acc + w[g->cidx[j]] * v;
            }
            dst[(i0 * n1 + i1) * n2 + i2] = acc;
        }
    }
}

int oracle_run_u32(int d, int r, int pattern, const int64_t *n, const uint32_t *w, int bkind, uint32_t bval,
                   const uint32_t *u0, int64_t T, uint32_t *uT)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !w || !u0 || !uT || T < 0) return -1;
    int64_t N = g.n[0] * g.n[1] * g.n[2];
    uint32_t *a = (uint32_t *)malloc(sizeof(uint32_t) * N), *b = (uint32_t *)malloc(sizeof(uint32_t) * N);
    if (!a || !b) { free(a); free(b); return -2; }
    memcpy(a, u0, sizeof(uint32_t) * N);
    for (int64_t t = 0; t < T; ++t) { step_u32(&g, w, bval, a, b); uint32_t *s = a; a = b; b = s; }
    memcpy(uT, a, sizeof(uint32_t) * N);
    free(a); free(b);
    return 0;
}

/* ------------------------------------------------- single output points
 * u_T at chosen points, from the dependency cone only: the value at level t
 * is needed on a box of half-width r*(T - t) around the point (in the d
 * stencil dimensions).  Level-0 cells read u0 through the boundary rule;
 * later cells are computed by the same sum as above, except Dirichlet cells
 * outside the domain, which stay bval.  Cells are addressed by virtual
 * coordinates, so periodic wrap needs no special case. */

typedef struct { int64_t lo[3], ext[3]; } box3;

static int64_t box_size(const box3 *b) { return b->ext[0] * b->ext[1] * b->ext[2]; }

static int in_domain(const or_geom *g, int64_t i0, int64_t i1, int64_t i2)
{
    return i0 >= 0 && i0 < g->n[0] && i1 >= 0 && i1 < g->n[1] && i2 >= 0 && i2 < g->n[2];
}

static void cone_box(const or_geom *g, const int64_t *p, int64_t h, box3 *b)
{
    for (int a = 0; a < 3; ++a) {
        int64_t hh = (a >= 3 - g->d) ? h : 0;
        b->lo[a] = p[a] - hh;
        b->ext[a] = 2 * hh + 1;
    }
}

#define CONE_POINTS_BODY(TYPE, ZERO, ACC_STEP)                                                          \
    for (int64_t q = 0; q < npts; ++q) {                                                                \
        int64_t p[3] = { 0, 0, 0 };                                                                     \
        for (int a = 0; a < d; ++a) {                                                                   \
            p[3 - d + a] = pts[q * d + a];                                                              \
            if (p[3 - d + a] < 0 || p[3 - d + a] >= n[a]) { free(cur); free(nxt); return -1; }          \
        }                                                                                               \
        box3 bc; cone_box(&g, p, (int64_t)r * T, &bc);                                                  \
        for (int64_t i0 = 0; i0 < bc.ext[0]; ++i0)                                                      \
            for (int64_t i1 = 0; i1 < bc.ext[1]; ++i1)                                                  \
                for (int64_t i2 = 0; i2 < bc.ext[2]; ++i2) {                                            \
                    int64_t lin;                                                                        \
                    int ok = resolve(&g, bc.lo[0] + i0, bc.lo[1] + i1, bc.lo[2] + i2, &lin);            \
                    cur[(i0 * bc.ext[1] + i1) * bc.ext[2] + i2] = ok ? u0[lin] : bval;                  \
                }                                                                                       \
        for (int64_t t = 1; t <= T; ++t) {                                                              \
            box3 bn; cone_box(&g, p, (int64_t)r * (T - t), &bn);                                        \
            for (int64_t i0 = 0; i0 < bn.ext[0]; ++i0)                                                  \
                for (int64_t i1 = 0; i1 < bn.ext[1]; ++i1)                                              \
                    for (int64_t i2 = 0; i2 < bn.ext[2]; ++i2) {                                        \
                        int64_t v0 = bn.lo[0] + i0, v1 = bn.lo[1] + i1, v2 = bn.lo[2] + i2;             \
                        TYPE acc = ZERO;                                                                \
                        if (g.bkind == 0 && !in_domain(&g, v0, v1, v2)) {                               \
                            acc = bval;                                                                 \
                        } else {                                                                        \
                            for (int j = 0; j < g.np; ++j) {                                            \
                                int64_t c0 = v0 + g.off[j][0] - bc.lo[0];                               \
                                int64_t c1 = v1 + g.off[j][1] - bc.lo[1];                               \
                                int64_t c2 = v2 + g.off[j][2] - bc.lo[2];                               \
                                TYPE v = cur[(c0 * bc.ext[1] + c1) * bc.ext[2] + c2];                   \
                                ACC_STEP;                                                               \
                            }                                                                           \
                        }                                                                               \
                        nxt[(i0 * bn.ext[1] + i1) * bn.ext[2] + i2] = acc;                              \
                    }                                                                                   \
            TYPE *s = cur; cur = nxt; nxt = s; bc = bn;                                                 \
        }                                                                                               \
        out[q] = cur[0];                                                                                \
    }

int oracle_points_f64(int d, int r, int pattern, const int64_t *n, const double *w, int bkind, double bval,
                      const double *u0, int64_t T, int64_t npts, const int64_t *pts, double *out)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !w || !u0 || !pts || !out || T < 0 || npts < 0) return -1;
    box3 b0; int64_t z[3] = { 0, 0, 0 }; cone_box(&g, z, (int64_t)r * T, &b0);
    double *cur = (double *)malloc(sizeof(double) * box_size(&b0));
    double *nxt = (double *)malloc(sizeof(double) * box_size(&b0));
    if (!cur || !nxt) { free(cur); free(nxt); return -2; }
    CONE_POINTS_BODY(double, 0.0, acc = acc + w[g.cidx[j]] * v)
    free(cur); free(nxt);
    return 0;
}

int oracle_points_u32(int d, int r, int pattern, const int64_t *n, const uint32_t *w, int bkind, uint32_t bval,
                      const uint32_t *u0, int64_t T, int64_t npts, const int64_t *pts, uint32_t *out)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !w || !u0 || !pts || !out || T < 0 || npts < 0) return -1;
    box3 b0; int64_t z[3] = { 0, 0, 0 }; cone_box(&g, z, (int64_t)r * T, &b0);
    uint32_t *cur = (uint32_t *)malloc(sizeof(uint32_t) * box_size(&b0));
    uint32_t *nxt = (uint32_t *)malloc(sizeof(uint32_t) * box_size(&b0));
    if (!cur || !nxt) { free(cur); free(nxt); return -2; }
    CONE_POINTS_BODY(uint32_t, 0u, acc = acc + w[g.cidx[j]] * v)
    free(cur); free(nxt);
    return 0;
}

/* ---------------------------------------------------------------- adjoint
 * The sweep is u_{t+1} = A u_t + c, where A is the linear part of one step
 * and c the constant Dirichlet contribution.  Its transpose distributes each
 * lam[x] to the cells x + o with weight w_o: periodic cells wrap, Dirichlet
 * boundary cells are constants and receive nothing. */

static void tstep_f64(const or_geom *g, const double *w, const double *lam, double *out)
{
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
    memset(out, 0, sizeof(double) * n0 * n1 * n2);
    for (int64_t i0 = 0; i0 < n0; ++i0)
        for (int64_t i1 = 0; i1 < n1; ++i1)
            for (int64_t i2 = 0; i2 < n2; ++i2) {
                double l = lam[(i0 * n1 + i1) * n2 + i2];
                for (int j = 0; j < g->np; ++j) {
                    int64_t lin;
                    if (resolve(g, i0 + g->off[j][0], i1 + g->off[j][1], i2 + g->off[j][2], &lin))
                        out[lin] = out[lin] + w[g->cidx[j]] * l;
                }
            }
}

int oracle_transpose_step_f64(int d, int r, int pattern, const int64_t *n, const double *w, int bkind,
                              const double *lam_in, double *lam_out)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !w || !lam_in || !lam_out) return -1;
    tstep_f64(&g, w, lam_in, lam_out);
    return 0;
}

/* loss = 0.5 * sum (u_T - target)^2 after T steps from u0; returns the loss,
 * d loss / d u0 and d loss / d w (compact order).  All states are stored. */
int oracle_adjoint_f64(int d, int r, int pattern, const int64_t *n, const double *w, int bkind, double bval,
                       const double *u0, const double *target, int64_t T,
                       double *grad_u0, double *grad_w, double *loss)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !w || !u0 || !target || !grad_u0 || !grad_w || !loss || T < 0)
        return -1;
    const int64_t n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], N = n0 * n1 * n2;
    double *U = (double *)malloc(sizeof(double) * N * (T + 1));
    double *lam = (double *)malloc(sizeof(double) * N), *tmp = (double *)malloc(sizeof(double) * N);
    if (!U || !lam || !tmp) { free(U); free(lam); free(tmp); return -2; }
    memcpy(U, u0, sizeof(double) * N);
    for (int64_t t = 0; t < T; ++t) step_f64(&g, w, bval, U + t * N, U + (t + 1) * N);
    double L = 0.0;
    for (int64_t i = 0; i < N; ++i) { double e = U[T * N + i] - target[i]; L = L + 0.5 * e * e; lam[i] = e; }
    *loss = L;
    for (int j = 0; j < g.np; ++j) grad_w[j] = 0.0;
    for (int64_t t = T - 1; t >= 0; --t) {
        const double *Ut = U + t * N;
        /* d u_{t+1}[x] / d w_o = u_t(x + o), boundary values included */
        for (int64_t i0 = 0; i0 < n0; ++i0)
            for (int64_t i1 = 0; i1 < n1; ++i1)
                for (int64_t i2 = 0; i2 < n2; ++i2) {
                    double l = lam[(i0 * n1 + i1) * n2 + i2];
                    for (int j = 0; j < g.np; ++j) {
                        int64_t lin;
                        double v = resolve(&g, i0 + g.off[j][0], i1 + g.off[j][1], i2 + g.off[j][2], &lin) ? Ut[lin] : bval;
                        grad_w[g.cidx[j]] = grad_w[g.cidx[j]] + l * v;
                    }
                }
        tstep_f64(&g, w, lam, tmp);
        double *s = lam; lam = tmp; tmp = s;
    }
    memcpy(grad_u0, lam, sizeof(double) * N);
    free(U); free(lam); free(tmp);
    return 0;
}

/* ------------------------------------------- variable coefficients
 * The same sweep with a coefficient per offset and per grid point (not in
 * the paper; the variable-coefficient form of the Section 1 definition):
 *     u_{t+1}[x] = sum_o c_o[x] * u_t(x + o),
 * c stored offset-major in compact order: c[j * N + x] for the j-th compact
 * offset.  Same boundary rule, same summation order. */

static void step_vc_f64(const or_geom *g, const double *c, double bval, const double *src, double *dst)
{
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2], N = n0 * n1 * n2;
    int64_t rows = n0 * n1;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t i0 = row / n1, i1 = row % n1;
        for (int64_t i2 = 0; i2 < n2; ++i2) {
            const int64_t x = (i0 * n1 + i1) * n2 + i2;
            double acc = 0.0;
            for (int j = 0; j < g->np; ++j) {
                int64_t lin;
                double v = resolve(g, i0 + g->off[j][0], i1 + g->off[j][1], i2 + g->off[j][2], &lin) ? src[lin] : bval;
                acc = acc + c[(int64_t)g->cidx[j] * N + x] * v;
            }
            dst[x] = acc;
        }
    }
}

int oracle_run_vc_f64(int d, int r, int pattern, const int64_t *n, const double *c, int bkind, double bval,
                      const double *u0, int64_t T, double *uT)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !c || !u0 || !uT || T < 0) return -1;
    int64_t N = g.n[0] * g.n[1] * g.n[2];
    double *a = (double *)malloc(sizeof(double) * N), *b = (double *)malloc(sizeof(double) * N);
    if (!a || !b) { free(a); free(b); return -2; }
    memcpy(a, u0, sizeof(double) * N);
    for (int64_t t = 0; t < T; ++t) { step_vc_f64(&g, c, bval, a, b); double *s = a; a = b; b = s; }
    memcpy(uT, a, sizeof(double) * N);
    free(a); free(b);
    return 0;
}

static void step_vc_u32(const or_geom *g, const uint32_t *c, uint32_t bval, const uint32_t *src, uint32_t *dst)
{
    const int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2], N = n0 * n1 * n2;
    int64_t rows = n0 * n1;
#pragma omp parallel for schedule(static)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t i0 = row / n1, i1 = row % n1;
        for (int64_t i2 = 0; i2 < n2; ++i2) {
            const int64_t x = (i0 * n1 + i1) * n2 + i2;
            uint32_t acc = 0u;
            for (int j = 0; j < g->np; ++j) {
                int64_t lin;
                uint32_t v = resolve(g, i0 + g->off[j][0], i1 + g->off[j][1], i2 + g->off[j][2], &lin) ? src[lin] : bval;
                acc = acc + c[(int64_t)g->cidx[j] * N + x] * v;
            }
            dst[x] = acc;
        }
    }
}

int oracle_run_vc_u32(int d, int r, int pattern, const int64_t *n, const uint32_t *c, int bkind, uint32_t bval,
                      const uint32_t *u0, int64_t T, uint32_t *uT)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !c || !u0 || !uT || T < 0) return -1;
    int64_t N = g.n[0] * g.n[1] * g.n[2];
    uint32_t *a = (uint32_t *)malloc(sizeof(uint32_t) * N), *b = (uint32_t *)malloc(sizeof(uint32_t) * N);
    if (!a || !b) { free(a); free(b); return -2; }
    memcpy(a, u0, sizeof(uint32_t) * N);
    for (int64_t t = 0; t < T; ++t) { step_vc_u32(&g, c, bval, a, b); uint32_t *s = a; a = b; b = s; }
    memcpy(uT, a, sizeof(uint32_t) * N);
    free(a); free(b);
    return 0;
}

/* loss = 0.5 * sum (u_T - target)^2 of the variable-coefficient sweep;
 * returns the loss, d loss / d u0 and d loss / d c (same layout as c):
 *     d loss / d c_o[x] = sum_t lam_{t+1}[x] * u_t(x + o)   (boundary values included)
 *     lam_t[y] = sum over (x, o) with x + o resolving to y of c_o[x] lam_{t+1}[x]. */
int oracle_adjoint_vc_f64(int d, int r, int pattern, const int64_t *n, const double *c, int bkind, double bval,
                          const double *u0, const double *target, int64_t T,
                          double *grad_u0, double *grad_c, double *loss)
{
    or_geom g;
    if (or_setup(&g, d, r, pattern, n, bkind) || !c || !u0 || !target || !grad_u0 || !grad_c || !loss || T < 0)
        return -1;
    const int64_t n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], N = n0 * n1 * n2;
    double *U = (double *)malloc(sizeof(double) * N * (T + 1));
    double *lam = (double *)malloc(sizeof(double) * N), *tmp = (double *)malloc(sizeof(double) * N);
    if (!U || !lam || !tmp) { free(U); free(lam); free(tmp); return -2; }
    memcpy(U, u0, sizeof(double) * N);
    for (int64_t t = 0; t < T; ++t) step_vc_f64(&g, c, bval, U + t * N, U + (t + 1) * N);
    double L = 0.0;
    for (int64_t i = 0; i < N; ++i) { double e = U[T * N + i] - target[i]; L = L + 0.5 * e * e; lam[i] = e; }
    *loss = L;
    for (int64_t i = 0; i < (int64_t)g.np * N; ++i) grad_c[i] = 0.0;
    for (int64_t t = T - 1; t >= 0; --t) {
        const double *Ut = U + t * N;
        memset(tmp, 0, sizeof(double) * N);
        for (int64_t i0 = 0; i0 < n0; ++i0)
            for (int64_t i1 = 0; i1 < n1; ++i1)
                for (int64_t i2 = 0; i2 < n2; ++i2) {
                    const int64_t x = (i0 * n1 + i1) * n2 + i2;
                    double l = lam[x];
                    for (int j = 0; j < g.np; ++j) {
                        int64_t lin;
                        const int64_t cj = (int64_t)g.cidx[j] * N + x;
                        if (resolve(&g, i0 + g.off[j][0], i1 + g.off[j][1], i2 + g.off[j][2], &lin)) {
                            grad_c[cj] = grad_c[cj] + l * Ut[lin];
                            tmp[lin] = tmp[lin] + c[cj] * l;
                        } else {
                            grad_c[cj] = grad_c[cj] + l * bval;
                        }
                    }
                }
        double *s = lam; lam = tmp; tmp = s;
    }
    memcpy(grad_u0, lam, sizeof(double) * N);
    free(U); free(lam); free(tmp);
    return 0;
}

/* ------------------------------------------------------------ reductions */

int oracle_sum_f64(int64_t N, const double *u, double *out)
{
    if (!u || !out || N < 0) return -1;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s = s + u[i];
    *out = s;
    return 0;
}

int oracle_sumsq_f64(int64_t N, const double *u, double *out)
{
    if (!u || !out || N < 0) return -1;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s = s + u[i] * u[i];
    *out = s;
    return 0;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
