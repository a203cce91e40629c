// tiling_check.cu -- host-only check of the tile geometry the fused and
// persistent kernels use (f2_tiling in k_fused2d.cuh, f3_lz in k_fused3d.cuh):
// column bands and row chunks (z ranges) must cover each axis exactly once --
// every row or plane in exactly one tile, the last one possibly shorter --
// and tiles must keep the minimum lengths the kernels assume (max(4 r k, 16)
// rows in 2D, max(4 r k, 8) planes in 3D, unless the axis itself is
// shorter); an explicit tile length is honoured within those bounds.
// Prints "ok <cases>" and exits 0, or the first failing case and exits 1.
#include <cstdio>

#include "k_fused2d.cuh"
#include "k_fused3d.cuh"

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
    std::printf("ok %lld\n", cases);
    return 0;
}
