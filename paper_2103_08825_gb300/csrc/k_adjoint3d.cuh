// k_adjoint3d.cuh -- one transposed step of a 3D sweep, streamed along z.
//
// Not in the paper (its method is a forward sweep; the derivative is this
// library's extension).  For lam = lam_{t+1} and u = u_t it computes
//     lam_t[x] = sum_o w_o lam[x - o]           (A^T lam; lam = 0 outside a Dirichlet domain)
//     gw_o    += sum_x lam[x] u(x + o)          (u = the boundary value outside)
// over the x of the grid, with the o in lexicographic order for lam_t -- the
// order the one-step adjoint kernels use, so its lam is bit-identical to
// theirs.
//
// A CTA owns 128 x 16 output columns x rows and a contiguous range of planes
// (the grid's tile-planes are split evenly over the resident CTAs, two per
// SM at radius 1).  The planes of lam and u, each with an x halo of 4 columns
// and a y halo of r rows, pass through a ring of 2r + 3 shared-memory slots
// filled by 16-byte cp.async copies (indices wrapped on periodic axes,
// outside values filled on Dirichlet ones; each thread's copies are resolved
// once per job), two planes ahead of the plane being computed; every grid
// element is read from HBM once per pass (plus the halos: a 4-column x halo
// costs whole DRAM sectors, so tiles are wide).  Each thread owns 4 x-points
// of 2 rows; a warp spans a tile row.  Weight-gradient terms: FP32 per thread over two
// planes (16 products per weight), an FP32 warp tree, then FP64 per warp in
// shared memory across all planes of the launch, and a fixed-order FP64 sum
// over warps into the CTA's partial slot -- deterministic for a given grid.
#pragma once

#include "common.cuh"

namespace sg {

constexpr int A3_THREADS = 256, A3_LX = 32;           // lanes along x: a whole warp spans a tile row
constexpr int A3_TX = 4 * A3_LX, A3_RY = 2;             // tile columns; rows per thread
constexpr int A3_TY = (A3_THREADS / A3_LX) * A3_RY;     // tile rows
constexpr int A3_XH = 4, A3_XW = A3_TX + 2 * A3_XH;
constexpr int A3_PF = 2;   // planes in flight ahead of the ones in use

struct Adj3Params {
    const float *lam_in;   // lam_{t+1}
    const float *u;        // u_t
    float *lam_out;        // lam_t
    double *partials;      // [gridDim.x][np]
    int nx, ny, nz;        // innermost first
    int tiles_x, tiles_y;
    int periodic;
    float bval;
    int first;             // 1: overwrite partials, 0: add
    int vec;               // nx % 4 == 0 and 16-byte aligned grids: 16-byte copies
    float w[kMaxPts];      // evaluation (lexicographic) order
};

template <int R> struct A3Geo {
    static constexpr int ROWS = A3_TY + 2 * R;
    static constexpr int SLOT = ROWS * A3_XW;                  // floats per plane slot
    static constexpr int NSL = 2 * R + 1 + A3_PF;              // 2r + 1 planes in use, A3_PF in flight
    static constexpr int SMEM = 2 * NSL * SLOT * 4;            // lam ring, u ring
};

// One plane z (virtual) of one grid into a slot: rows y0 - r .. y0 + TY + r - 1,
// columns x0 - XH .. x0 + TX + XH - 1; `fill` outside a Dirichlet domain.
template <int R>
__device__ __forceinline__ void a3_load_plane(float *slot, const float *__restrict__ g, const Adj3Params &p, int x0,
                                              int y0, int z, float fill) {
    constexpr int CH = A3_XW / 4;   // 16-byte chunks per row
    const bool periodic = p.periodic != 0;
    bool zin = z >= 0 && z < p.nz;
    if (!zin && periodic) { z = (int)wrap_idx(z, p.nz); zin = true; }
    for (int e = threadIdx.x; e < A3Geo<R>::ROWS * CH; e += A3_THREADS) {
        const int row = e / CH, c = e - row * CH;
        int y = y0 - R + row;
        bool yin = y >= 0 && y < p.ny;
        if (!yin && periodic) { y = (int)wrap_idx(y, p.ny); yin = true; }
        float *d = slot + row * A3_XW + 4 * c;
        const int x = x0 - A3_XH + 4 * c;
        if (!(zin && yin)) {
            d[0] = d[1] = d[2] = d[3] = fill;
            continue;
        }
        const float *rp = g + ((size_t)z * p.ny + y) * p.nx;
        if (p.vec) {
            // whole chunks: inside, one extent away (periodic) or outside
            int xs = x;
            bool xin = x >= 0 && x + 4 <= p.nx;
            if (!xin && periodic) {
                xs = x < 0 ? x + p.nx : x - p.nx;
                xin = xs >= 0 && xs + 4 <= p.nx;
            }
            if (xin) {
                cp_async16(d, rp + xs);
                continue;
            }
            if (!periodic) {
                d[0] = d[1] = d[2] = d[3] = fill;
                continue;
            }
        }
        // element by element (unaligned rows, or wrapping by more than one extent)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int xx = x + q;
            if (xx >= 0 && xx < p.nx) d[q] = __ldg(rp + xx);
            else if (periodic) d[q] = __ldg(rp + wrap_idx(xx, p.nx));
            else d[q] = fill;
        }
    }
}

// The same copy with each thread's chunks resolved once per job: soff[i] is
// the chunk's slot offset, goff[i] its element offset within a plane (-1: the
// fill value; -2: no chunk), so that a plane costs a few instructions per chunk.
// Used where rows are 16-byte multiples and every plane has < 2^31 elements.
template <int R, int NC>
__device__ __forceinline__ void a3_chunks(const Adj3Params &p, int x0, int y0, int (&soff)[NC], int (&goff)[NC]) {
    constexpr int CH = A3_XW / 4;
    const bool periodic = p.periodic != 0;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        const int e = threadIdx.x + i * A3_THREADS;
        soff[i] = 0;
        goff[i] = -2;
        if (e >= A3Geo<R>::ROWS * CH) continue;
        const int row = e / CH, c = e - row * CH;
        soff[i] = row * A3_XW + 4 * c;
        int y = y0 - R + row;
        bool yin = y >= 0 && y < p.ny;
        if (!yin && periodic) { y = (int)wrap_idx(y, p.ny); yin = true; }
        int x = x0 - A3_XH + 4 * c;
        bool xin = x >= 0 && x + 4 <= p.nx;
        if (!xin && periodic) {
            x = (int)wrap_idx(x, p.nx);   // whole chunks: nx is a multiple of 4
            xin = true;
        }
        goff[i] = (yin && xin) ? y * p.nx + x : -1;
    }
}

template <int NC>
__device__ __forceinline__ void a3_load_fast(float *slot, const float *__restrict__ g, const Adj3Params &p, int z,
                                             float fill, const int (&soff)[NC], const int (&goff)[NC]) {
    bool zin = z >= 0 && z < p.nz;
    if (!zin && p.periodic) { z = (int)wrap_idx(z, p.nz); zin = true; }
    const float *pl = g + (size_t)z * p.ny * p.nx;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        if (goff[i] == -2) continue;
        float *d = slot + soff[i];
        if (zin && goff[i] >= 0) cp_async16(d, pl + goff[i]);
        else *reinterpret_cast<float4 *>(d) = make_float4(fill, fill, fill, fill);
    }
}

__device__ __forceinline__ void a3_ld4(const float *p, float (&r)[4]) {
    const float4 m = *reinterpret_cast<const float4 *>(p);
    r[0] = m.x; r[1] = m.y; r[2] = m.z; r[3] = m.w;
}

// 12 values of a slot row around a thread's 4 columns: r[i] = column xl - 4 + i
// (NEEDX), else only r[4..7]
template <bool NEEDX>
__device__ __forceinline__ void a3_row(const float *rowp, float (&r)[12]) {
    const float4 m = *reinterpret_cast<const float4 *>(rowp);
    r[4] = m.x; r[5] = m.y; r[6] = m.z; r[7] = m.w;
    if constexpr (NEEDX) {
        const float4 a = *reinterpret_cast<const float4 *>(rowp - 4);
        const float4 b = *reinterpret_cast<const float4 *>(rowp + 4);
        r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
        r[8] = b.x; r[9] = b.y; r[10] = b.z; r[11] = b.w;
    }
}

template <int R, int PAT>
__global__ void __launch_bounds__(A3_THREADS, 2) adjoint3d_kernel(const __grid_constant__ Adj3Params p) {
    using Sh = Shape<3, R, PAT>;
    using G = A3Geo<R>;
    constexpr int NP = Sh::npts, NSL = G::NSL, SLOT = G::SLOT;
    constexpr int NC = (G::ROWS * (A3_XW / 4) + A3_THREADS - 1) / A3_THREADS;   // chunks a thread copies
    const bool fast = p.vec && (int64_t)p.ny * p.nx < (1ll << 31);
    extern __shared__ __align__(16) float a3_smem[];
    float *lam_ring = a3_smem, *u_ring = a3_smem + NSL * SLOT;
    __shared__ double gacc[A3_THREADS / 32][NP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hw = (warp * 32 + lane) / A3_LX;   // row group: tile rows A3_RY hw ..
    const int xl = (lane % A3_LX) * 4;
    for (int i = threadIdx.x; i < (A3_THREADS / 32) * NP; i += A3_THREADS) (&gacc[0][0])[i] = 0.0;
    float gw[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) gw[j] = 0.f;
    // this CTA's share of the tile-planes, in tile-major order
    const int64_t units = (int64_t)p.tiles_x * p.tiles_y * p.nz;
    int64_t u = units * blockIdx.x / gridDim.x;
    const int64_t uend = units * (blockIdx.x + 1) / gridDim.x;
    int nplanes_done = 0;   // planes since the last FP64 flush
    float lamC[3][A3_RY][4], uC[3][A3_RY][4];   // the 7-point star's centre rows of planes z - 1 .. z + 1
    while (u < uend) {
        const int tile = (int)(u / p.nz), z0 = (int)(u % p.nz);
        const int64_t zend = z0 + (uend - u);
        const int z1 = zend < p.nz ? (int)zend : p.nz;
        u += z1 - z0;
        const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
        const int x0 = tx * A3_TX, y0 = ty * A3_TY;
        const int nout = z1 - z0, nin = nout + 2 * R;   // input planes z0 - r .. z1 + r - 1
        int soff[NC], goff[NC];
        if (fast) a3_chunks<R, NC>(p, x0, y0, soff, goff);
        auto load = [&](int q) {   // input plane q of the job into its slot
            float *ls = lam_ring + (q % NSL) * SLOT, *us = u_ring + (q % NSL) * SLOT;
            if (fast) {
                a3_load_fast<NC>(ls, p.lam_in, p, z0 - R + q, 0.f, soff, goff);
                a3_load_fast<NC>(us, p.u, p, z0 - R + q, p.bval, soff, goff);
            } else {
                a3_load_plane<R>(ls, p.lam_in, p, x0, y0, z0 - R + q, 0.f);
                a3_load_plane<R>(us, p.u, p, x0, y0, z0 - R + q, p.bval);
            }
        };
        // prologue: input planes 0 .. NSL - 2, one copy group each
        for (int q = 0; q < NSL - 1; ++q) {
            if (q < nin) load(q);
            cp_async_commit();
        }
        for (int t = 0; t < nout; ++t) {
            // input planes t .. t + 2r landed (the A3_PF - 1 later groups may be pending)
            cp_async_wait<A3_PF - 1>();
            __syncthreads();
            {
                // refill the slot of plane t - 1, which every thread has finished with
                const int q = t + NSL - 1;
                if (q < nin) load(q);
                cp_async_commit();
            }
            const int z = z0 + t;
            if constexpr (PAT == STENCIL_STAR && R == 1) {
                // The 7-point star: centre rows of planes z - 1, z, z + 1 stay
                // in registers (C[0..2], rotated one plane per step, so each
                // plane's centre rows are read from shared memory once); the
                // rows above and below come from the slot, x-neighbours by
                // shuffles (the row's edge lanes read the slot's halo
                // columns).
                const int rbase = (hw * A3_RY + R) * A3_XW + A3_XH + xl;   // own first row in a slot
                if (t == 0) {
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int b = 0; b < A3_RY; ++b) {
                            a3_ld4(lam_ring + ((t + q) % NSL) * SLOT + rbase + b * A3_XW, lamC[q][b]);
                            a3_ld4(u_ring + ((t + q) % NSL) * SLOT + rbase + b * A3_XW, uC[q][b]);
                        }
                }
#pragma unroll
                for (int b = 0; b < A3_RY; ++b) {
                    a3_ld4(lam_ring + ((t + 2) % NSL) * SLOT + rbase + b * A3_XW, lamC[2][b]);
                    a3_ld4(u_ring + ((t + 2) % NSL) * SLOT + rbase + b * A3_XW, uC[2][b]);
                }
                const float *lz = lam_ring + ((t + 1) % NSL) * SLOT + rbase;
                const float *uz = u_ring + ((t + 1) % NSL) * SLOT + rbase;
                float lup[4], ldn[4], uup[4], udn[4];
                a3_ld4(lz - A3_XW, lup);
                a3_ld4(lz + A3_RY * A3_XW, ldn);
                a3_ld4(uz - A3_XW, uup);
                a3_ld4(uz + A3_RY * A3_XW, udn);
                float lL[A3_RY], lR[A3_RY], uL[A3_RY], uR[A3_RY];
#pragma unroll
                for (int b = 0; b < A3_RY; ++b) {
                    lL[b] = __shfl_up_sync(0xffffffffu, lamC[1][b][3], 1, A3_LX);
                    lR[b] = __shfl_down_sync(0xffffffffu, lamC[1][b][0], 1, A3_LX);
                    uL[b] = __shfl_up_sync(0xffffffffu, uC[1][b][3], 1, A3_LX);
                    uR[b] = __shfl_down_sync(0xffffffffu, uC[1][b][0], 1, A3_LX);
                    if (lane % A3_LX == 0) {
                        lL[b] = lz[b * A3_XW - 1];
                        uL[b] = uz[b * A3_XW - 1];
                    }
                    if (lane % A3_LX == A3_LX - 1) {
                        lR[b] = lz[b * A3_XW + 4];
                        uR[b] = uz[b * A3_XW + 4];
                    }
                }
                // the value at (plane z + dz, row b + dy, column v + dx)
                auto at = [&](const float (&Cc)[3][A3_RY][4], const float (&up)[4], const float (&dn)[4],
                              const float (&L)[A3_RY], const float (&Rr)[A3_RY], int b, int dz, int dy, int dx,
                              int v) -> float {
                    if (dz != 0) return Cc[1 + dz][b][v];
                    if (dy != 0) {
                        const int bb = b + dy;
                        return bb < 0 ? up[v] : (bb >= A3_RY ? dn[v] : Cc[1][bb][v]);
                    }
                    const int vv = v + dx;
                    return vv < 0 ? L[b] : (vv >= 4 ? Rr[b] : Cc[1][b][vv]);
                };
#pragma unroll
                for (int b = 0; b < A3_RY; ++b) {
                    const int y = y0 + hw * A3_RY + b, xg = x0 + xl;
                    float lc[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) lc[v] = (y < p.ny && xg + v < p.nx) ? lamC[1][b][v] : 0.f;
                    float acc[4];
                    bool first = true;
#pragma unroll
                    for (int oz = -R; oz <= R; ++oz)
#pragma unroll
                        for (int oy = -R; oy <= R; ++oy)
#pragma unroll
                            for (int ox = -R; ox <= R; ++ox) {
                                if (!Sh::inc(oz, oy, ox)) continue;
                                const int j = Sh::widx(oz, oy, ox);
                                const float w = p.w[j];
#pragma unroll
                                for (int v = 0; v < 4; ++v) {
                                    const float l = at(lamC, lup, ldn, lL, lR, b, -oz, -oy, -ox, v);   // lam(x - o)
                                    acc[v] = first ? __fmul_rn(w, l) : __fmaf_rn(w, l, acc[v]);
                                    gw[j] = __fmaf_rn(lc[v], at(uC, uup, udn, uL, uR, b, oz, oy, ox, v), gw[j]);
                                }
                                first = false;
                            }
                    if (y < p.ny) {
                        float *out = p.lam_out + ((size_t)z * p.ny + y) * p.nx + xg;
                        if (p.vec && xg + 4 <= p.nx) {
                            *reinterpret_cast<float4 *>(out) = make_float4(acc[0], acc[1], acc[2], acc[3]);
                        } else {
#pragma unroll
                            for (int v = 0; v < 4; ++v)
                                if (xg + v < p.nx) out[v] = acc[v];
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                    for (int b = 0; b < A3_RY; ++b)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            lamC[q][b][v] = lamC[q + 1][b][v];
                            uC[q][b][v] = uC[q + 1][b][v];
                        }
            } else {
    #pragma unroll
                for (int b = 0; b < A3_RY; ++b) {
                    const int yl = hw * A3_RY + b;        // tile row
                    const int y = y0 + yl, xg = x0 + xl;
                    const int rowoff = (yl + R) * A3_XW + A3_XH + xl;
                    // lam at this thread's own points; 0 for points outside the grid
                    float lc[4];
                    {
                        const float4 m = *reinterpret_cast<const float4 *>(lam_ring + ((t + R) % NSL) * SLOT + rowoff);
                        lc[0] = m.x; lc[1] = m.y; lc[2] = m.z; lc[3] = m.w;
                        const bool yin = y < p.ny;
    #pragma unroll
                        for (int v = 0; v < 4; ++v) lc[v] = (yin && xg + v < p.nx) ? lc[v] : 0.f;
                    }
                    float acc[4];
                    bool first = true;
    #pragma unroll
                    for (int oz = -R; oz <= R; ++oz) {
                        const float *ls = lam_ring + ((t + R - oz) % NSL) * SLOT;   // plane z - oz
                        const float *us = u_ring + ((t + R + oz) % NSL) * SLOT;     // plane z + oz
    #pragma unroll
                        for (int oy = -R; oy <= R; ++oy) {
                            bool any = false;
    #pragma unroll
                            for (int ox = -R; ox <= R; ++ox) any = any || Sh::inc(oz, oy, ox);
                            if (!any) continue;
                            float lr[12], ur[12];
                            if (PAT == STENCIL_BOX || (oz == 0 && oy == 0)) {
                                a3_row<true>(ls + rowoff - oy * A3_XW, lr);
                                a3_row<true>(us + rowoff + oy * A3_XW, ur);
                            } else {
                                a3_row<false>(ls + rowoff - oy * A3_XW, lr);
                                a3_row<false>(us + rowoff + oy * A3_XW, ur);
                            }
    #pragma unroll
                            for (int ox = -R; ox <= R; ++ox) {
                                if (!Sh::inc(oz, oy, ox)) continue;
                                const int j = Sh::widx(oz, oy, ox);
                                const float w = p.w[j];
    #pragma unroll
                                for (int v = 0; v < 4; ++v) {
                                    const float l = lr[4 + v - ox];   // lam(x - o)
                                    acc[v] = first ? __fmul_rn(w, l) : __fmaf_rn(w, l, acc[v]);
                                    gw[j] = __fmaf_rn(lc[v], ur[4 + v + ox], gw[j]);   // lam(x) u(x + o)
                                }
                                first = false;
                            }
                        }
                    }
                    if (y < p.ny) {
                        float *out = p.lam_out + ((size_t)z * p.ny + y) * p.nx + xg;
                        if (p.vec && xg + 4 <= p.nx) {
                            *reinterpret_cast<float4 *>(out) = make_float4(acc[0], acc[1], acc[2], acc[3]);
                        } else {
    #pragma unroll
                            for (int v = 0; v < 4; ++v)
                                if (xg + v < p.nx) out[v] = acc[v];
                        }
                    }
                }
            }
            // every two planes: FP32 warp tree, FP64 per warp (fixed order)
            if (++nplanes_done == 2) {
                nplanes_done = 0;
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    float s = gw[j];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) gacc[warp][j] += (double)s;
                    gw[j] = 0.f;
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();   // the next job's prologue overwrites the ring
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        float s = gw[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) gacc[warp][j] += (double)s;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double s = 0.0;
        for (int wi = 0; wi < A3_THREADS / 32; ++wi) s += gacc[wi][threadIdx.x];
        double *dst = p.partials + (size_t)blockIdx.x * NP + threadIdx.x;
        *dst = p.first ? s : *dst + s;
    }
}

}  // namespace sg
