// k_plain.cuh -- one Jacobi step per launch (the plain GPU sweep).
//
// Every thread produces 4 consecutive points of one x-row.  For each row
// offset (o_0, o_1) it reads the span of the source row it needs (x-halo of
// r only for the rows where the pattern has x-offsets), straight from HBM/L2
// through the read-only path, then accumulates the offsets in lexicographic
// order (paper, Section 1: the point update is a weighted sum of neighbours
// at the previous time level).  This is the GPU analogue of the paper's
// "multiple load" vectorisation (Section 2.1): each output loads all of its
// own inputs, and neighbour reuse is left to the caches.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "plan.h"

namespace sg {

template <typename S, typename C>
__device__ __forceinline__ void ldg4(const S *p, C out[4]) {
    if constexpr (sizeof(S) == 4) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const S *s = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = to_c(s[i]);
    } else if constexpr (sizeof(S) == 8) {
        uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
        uint4 b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
        const S *sa = reinterpret_cast<const S *>(&a);
        const S *sb = reinterpret_cast<const S *>(&b);
        out[0] = to_c(sa[0]); out[1] = to_c(sa[1]); out[2] = to_c(sb[0]); out[3] = to_c(sb[1]);
    } else {
        uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        const S *s = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = to_c(s[i]);
    }
}

template <typename S, typename C>
__device__ __forceinline__ void st4(S *p, const C in[4]) {
    S tmp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tmp[i] = from_c<S>(in[i]);
    if constexpr (sizeof(S) == 4) {
        *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(tmp);
    } else if constexpr (sizeof(S) == 8) {
        reinterpret_cast<uint4 *>(p)[0] = reinterpret_cast<const uint4 *>(tmp)[0];
        reinterpret_cast<uint4 *>(p)[1] = reinterpret_cast<const uint4 *>(tmp)[1];
    } else {
        *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(tmp);
    }
}

// One 4-point group of row (i0, i1) starting at x0.  INNER: the whole
// neighbourhood lies inside the grid, so no boundary logic runs.
template <int DT, int D, int R, int PAT, bool INNER>
__device__ __forceinline__ void plain_group(const PlainParams<typename Traits<DT>::C> &p,
                                            const typename Traits<DT>::S *__restrict__ src,
                                            typename Traits<DT>::S *__restrict__ dst, int64_t i0, int64_t i1,
                                            int64_t x0) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using Sh = Shape<D, R, PAT>;
    constexpr int VX = 4;
    const int64_t n0 = p.g.n0, n1 = p.g.n1, n2 = p.g.n2;
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    const C bval = p.g.bval;
    const S *centre = src + (i0 * n1 + i1) * n2;
    C acc[VX];
    bool first = true;
#pragma unroll
    for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz) {
#pragma unroll
        for (int oy = (D >= 2 ? -R : 0); oy <= (D >= 2 ? R : 0); ++oy) {
            if (!Sh::inc(oz, oy, 0)) continue;
            const bool halo = (PAT == STENCIL_BOX) || (oz == 0 && oy == 0);
            C span[VX + 2 * R];
            if constexpr (INNER) {
                const S *rowp = centre + ((int64_t)oz * n1 + oy) * n2;
                if (p.vec_ok) {
                    ldg4<S, C>(rowp + x0, span + R);
                } else {
#pragma unroll
                    for (int q = 0; q < VX; ++q) span[R + q] = to_c(__ldg(rowp + x0 + q));
                }
                if (halo) {
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        span[q] = to_c(__ldg(rowp + x0 - R + q));
                        span[R + VX + q] = to_c(__ldg(rowp + x0 + VX + q));
                    }
                }
            } else {
                int64_t r0 = i0 + oz, r1 = i1 + oy;
                bool row_ok = true;
                if (r0 < 0 || r0 >= n0) { if (periodic) r0 = wrap_idx(r0, n0); else row_ok = false; }
                if (r1 < 0 || r1 >= n1) { if (periodic) r1 = wrap_idx(r1, n1); else row_ok = false; }
                const S *rowp = src + (r0 * n1 + r1) * n2;
#pragma unroll
                for (int q = 0; q < VX + 2 * R; ++q) {
                    if (!halo && (q < R || q >= R + VX)) continue;
                    const int64_t x = x0 - R + q;
                    if (!row_ok) span[q] = bval;
                    else if (x >= 0 && x < n2) span[q] = to_c(__ldg(rowp + x));
                    else if (periodic) span[q] = to_c(__ldg(rowp + wrap_idx(x, n2)));
                    else span[q] = bval;
                }
            }
#pragma unroll
            for (int ox = -R; ox <= R; ++ox) {
                if (!Sh::inc(oz, oy, ox)) continue;
                const C w = p.w[Sh::widx(oz, oy, ox)];
#pragma unroll
                for (int v = 0; v < VX; ++v)
                    acc[v] = first ? op_mul(w, span[R + v + ox]) : op_fma(w, span[R + v + ox], acc[v]);
                first = false;
            }
        }
    }
    S *out = dst + (i0 * n1 + i1) * n2;
    if (p.vec_ok && x0 + VX <= n2) {
        st4<S, C>(out + x0, acc);
    } else {
#pragma unroll
        for (int v = 0; v < VX; ++v)
            if (x0 + v < n2) out[x0 + v] = from_c<S>(acc[v]);
    }
}

template <int DT, int D, int R, int PAT>
__global__ void __launch_bounds__(256) plain_kernel(const __grid_constant__ PlainParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    constexpr int VX = 4;
    const S *__restrict__ src = static_cast<const S *>(p.src);
    S *__restrict__ dst = static_cast<S *>(p.dst);
    const int64_t n0 = p.g.n0, n1 = p.g.n1, n2 = p.g.n2;
    const int64_t groups = (n2 + VX - 1) / VX;
    // grid: x over 4-point groups of a row, y over rows, z over planes
    for (int64_t i0 = blockIdx.z; i0 < n0; i0 += gridDim.z) {
        const bool z_in = D < 3 || (i0 >= R && i0 + R < n0);
        for (int64_t i1 = blockIdx.y; i1 < n1; i1 += gridDim.y) {
            const bool zy_in = z_in && (D < 2 || (i1 >= R && i1 + R < n1));
            for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
                 g += (int64_t)gridDim.x * blockDim.x) {
                const int64_t x0 = g * VX;
                if (zy_in && x0 - R >= 0 && x0 + VX + R <= n2)
                    plain_group<DT, D, R, PAT, true>(p, src, dst, i0, i1, x0);
                else
                    plain_group<DT, D, R, PAT, false>(p, src, dst, i0, i1, x0);
            }
        }
    }
}

// The one-step sweep for grids with moderate extents (every extent > 2r + 2,
// rows and planes addressable by the launch grid): one thread computes 4
// x-points of RB consecutive rows of one plane.  Row and plane indices are
// 32-bit and uniform across a warp's lanes, so rows outside the grid cost one
// uniform branch; each row used is addressed once (one 64-bit pointer), rows
// shared by the RB outputs are loaded once, and x-halo values at the grid's
// ends go through a predicated load (wrap by +-n, or the boundary value).
template <int DT, int D, int R, int PAT, int RB>
__global__ void __launch_bounds__(256) plain_rows_kernel(const __grid_constant__ PlainParams<typename Traits<DT>::C> p) {
    using S = typename Traits<DT>::S;
    using C = typename Traits<DT>::C;
    using Sh = Shape<D, R, PAT>;
    constexpr int VX = 4;
    constexpr int NZ = D == 3 ? 2 * R + 1 : 1;          // planes read
    constexpr int NY = D >= 2 ? RB + 2 * R : 1;         // rows read per plane
    const S *__restrict__ src = static_cast<const S *>(p.src);
    S *__restrict__ dst = static_cast<S *>(p.dst);
    const int n0 = (int)p.g.n0, n1 = (int)p.g.n1, n2 = (int)p.g.n2;
    const bool periodic = p.g.bkind == STENCIL_PERIODIC;
    const C bval = p.g.bval;
    const int i0 = blockIdx.z;
    const int i1b = (blockIdx.y * blockDim.y + threadIdx.y) * RB;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
    if (x0 >= n2 || i1b >= n1) return;
    const bool full = x0 + VX <= n2;
    C val[NZ][NY][VX + 2 * R];
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
            C *row = val[jz][jy];
            if (!ok) {
#pragma unroll
                for (int q = 0; q < VX + 2 * R; ++q) row[q] = bval;
                continue;
            }
            const S *rowp = src + ((int64_t)z * n1 + y) * n2;
            if (full && p.vec_ok) {
                ldg4<S, C>(rowp + x0, row + R);
            } else {
#pragma unroll
                for (int q = 0; q < VX; ++q) {   // last, partial group: wrap or boundary value
                    const int x = x0 + q;
                    row[R + q] = x < n2 ? to_c(__ldg(rowp + x)) : (periodic ? to_c(__ldg(rowp + x - n2)) : bval);
                }
            }
            if (halo) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    int xl = x0 - R + q, xr = x0 + VX + q;
                    const bool il = xl >= 0, ir = xr < n2;
                    xl = il ? xl : xl + n2;
                    xr = ir ? xr : xr - n2;
                    row[q] = (il || periodic) ? to_c(__ldg(rowp + xl)) : bval;
                    row[R + VX + q] = (ir || periodic) ? to_c(__ldg(rowp + xr)) : bval;
                }
            }
        }
    }
#pragma unroll
    for (int b = 0; b < RB; ++b) {
        const int yo = D >= 2 ? i1b + b : 0;
        if (yo >= n1) break;
        C acc[VX];
        bool first = true;
#pragma unroll
        for (int oz = (D == 3 ? -R : 0); oz <= (D == 3 ? R : 0); ++oz)
#pragma unroll
            for (int oy = (D >= 2 ? -R : 0); oy <= (D >= 2 ? R : 0); ++oy)
#pragma unroll
                for (int ox = -R; ox <= R; ++ox) {
                    if (!Sh::inc(oz, oy, ox)) continue;
                    const C w = p.w[Sh::widx(oz, oy, ox)];
                    const C *row = val[D == 3 ? oz + R : 0][D >= 2 ? R + b + oy : 0];
#pragma unroll
                    for (int v = 0; v < VX; ++v)
                        acc[v] = first ? op_mul(w, row[R + v + ox]) : op_fma(w, row[R + v + ox], acc[v]);
                    first = false;
                }
        S *out = dst + ((int64_t)i0 * n1 + yo) * n2;
        if (p.vec_ok && full) {
            st4<S, C>(out + x0, acc);
        } else {
#pragma unroll
            for (int v = 0; v < VX; ++v)
                if (x0 + v < n2) out[x0 + v] = from_c<S>(acc[v]);
        }
    }
}

template <typename C>
static void fill_geom(const stencil_plan_s &P, GridGeom<C> &g) {
    g.n0 = P.n[0];
    g.n1 = P.n[1];
    g.n2 = P.n[2];
    g.bkind = P.bkind;
    if constexpr (sizeof(C) == 4 && C(-1) > C(0)) {
        g.bval = (C)(uint32_t)(int64_t)P.bval;
    } else {
        g.bval = (C)P.bval;
    }
}

template <typename C>
static C conv_weight(double w) {
    if constexpr (sizeof(C) == 4 && C(-1) > C(0)) return (C)(uint32_t)(int64_t)w;  // uint32
    else return (C)w;
}

template <int DT, int D, int R, int PAT>
static cudaError_t launch_plain_t(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    using C = typename Traits<DT>::C;
    PlainParams<C> p;
    fill_geom<C>(P, p.g);
    p.src = src;
    p.dst = dst;
    p.np = P.np;
    p.vec_ok = (P.n[2] % 4 == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
    for (int j = 0; j < P.np; ++j) p.w[j] = conv_weight<C>(P.w_eval[j]);
    const int64_t groups = (P.n[2] + 3) / 4;
    int64_t bx = (groups + 255) / 256;
    if (bx > (1ll << 30)) bx = 1ll << 30;
    // two rows per thread where the loaded rows stay few (all but the 3D box)
    constexpr int RB = (D >= 2 && !(D == 3 && PAT == STENCIL_BOX)) ? 2 : 1;
    // block: TX threads along a row (the row's groups, up to 256), TY rows
    const int tx = (int)std::min<int64_t>(256, (groups + 31) / 32 * 32);
    const int ty = 256 / tx;
    const int64_t bxr = (groups + tx - 1) / tx;
    const int64_t rows = (P.n[1] + (int64_t)RB * ty - 1) / ((int64_t)RB * ty);
    // wrapping by one extent must land inside the grid; the launch grid must
    // cover every row and plane; 32-bit indices
    const bool big = (D < 3 || P.n[0] > 2 * R + 2) && (D < 2 || P.n[1] > 2 * R + RB + 2) && P.n[2] >= 2 * (4 + R) &&
                     P.n[0] <= 65535 && rows <= 65535 && P.n[2] < (1ll << 30) && P.n[1] < (1ll << 30);
    if (big) {
        const dim3 grid((unsigned)bxr, (unsigned)rows, (unsigned)P.n[0]);
        plain_rows_kernel<DT, D, R, PAT, RB><<<grid, dim3(tx, ty), 0, st>>>(p);
    } else {
        const dim3 grid((unsigned)bx, (unsigned)(P.n[1] < 65535 ? P.n[1] : 65535),
                        (unsigned)(P.n[0] < 65535 ? P.n[0] : 65535));
        plain_kernel<DT, D, R, PAT><<<grid, 256, 0, st>>>(p);
    }
    return cudaGetLastError();
}

template <int DT, int D>
static cudaError_t dispatch_r(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    const bool box = P.pattern == STENCIL_BOX;
    switch (P.r) {
        case 1: return box ? launch_plain_t<DT, D, 1, STENCIL_BOX>(P, src, dst, st)
                           : launch_plain_t<DT, D, 1, STENCIL_STAR>(P, src, dst, st);
        case 2: return box ? launch_plain_t<DT, D, 2, STENCIL_BOX>(P, src, dst, st)
                           : launch_plain_t<DT, D, 2, STENCIL_STAR>(P, src, dst, st);
        case 3: return box ? launch_plain_t<DT, D, 3, STENCIL_BOX>(P, src, dst, st)
                           : launch_plain_t<DT, D, 3, STENCIL_STAR>(P, src, dst, st);
    }
    return cudaErrorInvalidValue;
}

template <int DT>
cudaError_t plain_dispatch_d(const stencil_plan_s &P, const void *src, void *dst, cudaStream_t st) {
    switch (P.dim) {
        case 1: return dispatch_r<DT, 1>(P, src, dst, st);
        case 2: return dispatch_r<DT, 2>(P, src, dst, st);
        case 3: return dispatch_r<DT, 3>(P, src, dst, st);
    }
    return cudaErrorInvalidValue;
}

// one translation unit per storage type (k_plain_<dtype>.cu) instantiates
// plain_dispatch_d, so that the build compiles them in parallel
cudaError_t launch_plain_F64(const stencil_plan_s &, const void *, void *, cudaStream_t);
cudaError_t launch_plain_F32(const stencil_plan_s &, const void *, void *, cudaStream_t);
cudaError_t launch_plain_BF16(const stencil_plan_s &, const void *, void *, cudaStream_t);
cudaError_t launch_plain_F16(const stencil_plan_s &, const void *, void *, cudaStream_t);
cudaError_t launch_plain_I32(const stencil_plan_s &, const void *, void *, cudaStream_t);

}  // namespace sg
