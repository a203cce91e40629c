// tiling_check.cu -- host-only check of the tile geometry the fused and
// persistent kernels use (f2_tiling in k_fused2d.cuh, f3_lz in k_fused3d.cuh):
// column bands and row chunks (z ranges) must cover each axis exactly once --
// every row or plane in exactly one tile, the last one possibly shorter --
// and tiles must keep the minimum lengths the kernels assume (max(4 r k, 16)
// rows in 2D, max(4 r k, 8) planes in 3D, unless the axis itself is
// shorter); an explicit tile length is honoured within those bounds.  The x
// and y tiling of the 3D kernel (f3_axis, with the TMA path's narrower x halo
// f3_hx): outputs partition the axis, every window holds its outputs plus the
// r k halo (clipped at a Dirichlet domain's ends), Dirichlet windows stay in
// the domain, and on the TMA path every window starts on a 16-byte boundary
// (a TMA copy at an unaligned x raises an illegal-instruction fault).  The
// tessellation's closed-form level interval of a coordinate (tess_levels)
// against membership in the per-level ranges (tess_range).
// Prints "ok <cases>" and exits 0, or the first failing case and exits 1.
#include <cstdio>

#include "k_fused2d.cuh"
#include "k_fused3d.cuh"
#include "k_tess.cuh"

static bool cover(long long n, long long len, long long tiles) {
    return len >= 1 && tiles >= 1 && tiles * len >= n && (tiles - 1) * len < n;
}

int main() {
    long long cases = 0;
    const int bws[] = {2, 4, 56, 96, 112, 120, 124, 128};
    const long long slots_list[] = {1, 7, 608, 3040, 9728};
    for (long long nx : {1LL, 3LL, 37LL, 120LL, 121LL, 1000LL, 8192LL, 100003LL})
        for (long long ny : {1LL, 2LL, 15LL, 16LL, 17LL, 64LL, 333LL, 8192LL, 70001LL})
            for (int bw : bws)
                for (int rk = 1; rk <= 16; rk *= 2)
                    for (long long slots : slots_list)
                        for (int per_slot = 1; per_slot <= 3; ++per_slot)
                            for (int rows : {0, 1, 16, 17, 64, 5000}) {
                                const sg::F2Tiling t = sg::f2_tiling(nx, ny, bw, rk, slots, per_slot, rows);
                                const long long min_ly = 4 * rk > 16 ? 4 * rk : 16;
                                const long long want_min = min_ly < ny ? min_ly : ny;
                                bool ok = cover(nx, bw, t.bands) && cover(ny, t.Ly, t.chunks) && t.Ly >= want_min;
                                if (rows > 0) ok = ok && t.Ly == (rows > min_ly ? (rows < ny ? rows : ny) : want_min);
                                if (!ok) {
                                    std::printf("FAIL 2D nx=%lld ny=%lld bw=%d rk=%d slots=%lld per_slot=%d rows=%d: "
                                                "bands=%lld Ly=%lld chunks=%lld\n", nx, ny, bw, rk, slots, per_slot, rows,
                                                (long long)t.bands, (long long)t.Ly, (long long)t.chunks);
                                    return 1;
                                }
                                ++cases;
                            }
    for (long long nz : {1LL, 5LL, 8LL, 9LL, 31LL, 256LL, 512LL, 4097LL})
        for (long long tiles : {1LL, 10LL, 110LL, 5000LL})
            for (long long slots : {1LL, 152LL, 304LL})
                for (int rk = 1; rk <= 8; rk *= 2)
                    for (int lz : {0, 1, 8, 13, 64, 100000}) {
                        const long long l = sg::f3_lz(nz, tiles, slots, rk, lz);
                        const long long min_lz = 4 * rk > 8 ? 4 * rk : 8;
                        const long long want_min = min_lz < nz ? min_lz : nz;
                        const long long chunks = (nz + l - 1) / l;
                        bool ok = cover(nz, l, chunks) && l >= want_min && l <= nz;
                        if (lz > 0) ok = ok && l == (lz > min_lz ? (lz < nz ? lz : nz) : want_min);
                        if (!ok) {
                            std::printf("FAIL 3D nz=%lld tiles=%lld slots=%lld rk=%d lz=%d: Lz=%lld\n", nz, tiles, slots,
                                        rk, lz, l);
                            return 1;
                        }
                        ++cases;
                    }
    // 3D window tiling of one axis: W columns (window), AL elements per 16
    // bytes, halo h = f3_hx (TMA) or the AL-rounded halo (periodic / cp.async)
    const int geoms[][2] = {{32, 2}, {64, 4}, {64, 8}};   // FP64, FP32/int32, BF16/F16
    for (const auto &gm : geoms)
        for (int rk = 1; rk <= 4; ++rk)
            for (int tma = 0; tma <= 1; ++tma)
                for (int dir = 0; dir <= 1; ++dir) {
                    if (tma && !dir) continue;   // periodic grids never use TMA
                    const int W = gm[0], al = gm[1];
                    const int h = tma ? sg::f3_hx(rk, W, al) : (rk + al - 1) / al * al;
                    if (W - 2 * h < 1) continue;
                    for (long long n = 1; n <= 700; ++n) {
                        if (tma && n % al != 0) continue;   // TMA needs 16-byte rows
                        const sg::F3Axis a = sg::f3_axis(n, W, h, dir != 0);
                        long long next = 0;
                        bool ok = h >= rk;
                        for (int t = 0; t < a.T && ok; ++t) {
                            int os, oe, ws;
                            sg::f3_tile(a, t, os, oe, ws);
                            ok = os == next && oe > os && oe <= n;
                            next = oe;
                            const long long need_lo = dir ? (os - rk > 0 ? os - rk : 0) : os - rk;
                            const long long need_hi = dir ? (oe + rk < n ? oe + rk : n) : oe + rk;
                            ok = ok && ws <= need_lo && ws + W >= need_hi;
                            if (dir && n > W) ok = ok && ws >= 0 && ws + W <= n;
                            if (tma) ok = ok && ws % al == 0;
                        }
                        ok = ok && next == n;
                        if (!ok) {
                            std::printf("FAIL 3D axis W=%d al=%d rk=%d tma=%d dir=%d n=%lld h=%d\n", W, al, rk, tma,
                                        dir, n, h);
                            return 1;
                        }
                        ++cases;
                    }
                }
    // tess_levels: t in [lo, hi]  <=>  c in tess_range(t), for every in-domain c
    for (int periodic = 0; periodic <= 1; ++periodic)
        for (int n : {8, 9, 31, 64, 100})
            for (int b : {4, 8, 16, 32})
                for (int r = 1; r <= 3; ++r) {
                    sg::TessAxis ax{n, b < n ? b : n, 0, periodic};
                    ax.m = ax.n < 2 * ax.b ? 1 : ax.n / ax.b;
                    for (int inv = 0; inv <= 1; ++inv)
                        for (int i = 0; i < sg::tess_count(ax, inv != 0); ++i)
                            for (int c = -3 * b; c < n + 3 * b; ++c) {
                                int lo, hi;
                                sg::tess_levels(ax, inv != 0, i, c, r, lo, hi);
                                for (int t = 1; t <= 12; ++t) {
                                    int rl, rh;
                                    sg::tess_range(ax, inv != 0, i, t, r, rl, rh);
                                    const bool in_range = c >= rl && c < rh;
                                    const bool in_dom = periodic || (c >= 0 && c < n);
                                    if (!in_dom) continue;
                                    if (in_range != (t >= lo && t <= hi)) {
                                        std::printf("FAIL tess_levels n=%d b=%d r=%d periodic=%d inv=%d i=%d c=%d t=%d\n",
                                                    n, b, r, periodic, inv, i, c, t);
                                        return 1;
                                    }
                                    ++cases;
                                }
                            }
                }
    std::printf("ok %lld\n", cases);
    return 0;
}
