// tile_span_check.cu -- host-only check of tile_span (common.cuh), the
// dependency sets of the persistent multi-pass kernels: for every window
// [lo, hi) with -n <= lo < hi <= 2n, tile length and boundary kind, the tiles
// it lists (possibly repeated) must be exactly the tiles holding at least one
// coordinate of the window -- taken modulo n on a periodic axis, clipped to
// [0, n) otherwise -- and every listed index must lie in [0, tiles).  A
// missing tile would let a tile read data still being written; an extra or
// out-of-range one would wait on a counter that never advances.
// Prints "ok <cases>" and exits 0, or prints the first failing case and
// exits 1.  Needs no GPU.
#include <cstdio>
#include <set>

#include "common.cuh"

int main() {
    long long cases = 0;
    for (int n = 1; n <= 48; ++n)
        for (int len = 1; len <= n + 3; ++len) {
            const int tiles = (n + len - 1) / len;
            for (int per = 0; per < 2; ++per)
                for (int lo = -n; lo <= 2 * n; ++lo)
                    for (int hi = lo + 1; hi <= 2 * n; ++hi) {
                        std::set<int> want;
                        for (int x = lo; x < hi; ++x) {
                            int xx = x;
                            if (xx < 0 || xx >= n) {
                                if (!per) continue;
                                xx = ((xx % n) + n) % n;
                            }
                            want.insert(xx / len);
                        }
                        const sg::TileSpan s = sg::tile_span(lo, hi, n, len, per != 0);
                        std::set<int> got;
                        bool bad = s.n0 < 0 || s.n1 < 0 || s.n2 < 0;
                        for (int i = 0; i < s.count() && !bad; ++i) {
                            const int t = s.at(i);
                            if (t < 0 || t >= tiles) bad = true;
                            got.insert(t);
                        }
                        if (bad || got != want) {
                            std::printf("FAIL n=%d len=%d periodic=%d lo=%d hi=%d: %zu tiles expected, %zu listed%s\n",
                                        n, len, per, lo, hi, want.size(), got.size(), bad ? " (index out of range)" : "");
                            return 1;
                        }
                        ++cases;
                    }
        }
    std::printf("ok %lld\n", cases);
    return 0;
}
