// Host-side check of the membership search shared with the search kernels (search_util.h):
// against std::binary_search on sorted runs of distinct ids of many shapes, every key in the run
// and every gap between keys, and the step bound 2 * ceil(log2(L)) + 2 loads.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "search_util.h"

int main() {
    std::mt19937_64 rng(12345);
    long long checks = 0, fails = 0, max_over = 0;
    auto run = [&](std::vector<int32_t> v) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        const uint32_t L = (uint32_t)v.size();
        auto at = [&](uint32_t i) { return v[i]; };
        std::vector<int32_t> keys = {0, 1, 2147483646, 2147483647};
        for (int32_t x : v) {
            keys.push_back(x);
            if (x > 0) keys.push_back(x - 1);
            if (x < 2147483647) keys.push_back(x + 1);
        }
        const long long bound = 2 * (long long)std::ceil(std::log2((double)std::max<uint32_t>(L, 2))) + 2;
        for (int32_t c : keys) {
            // whole run and random sub-ranges
            for (int rep = 0; rep < 3; rep++) {
                uint32_t lo = 0, hi = L;
                if (rep && L) {
                    lo = (uint32_t)(rng() % (L + 1));
                    hi = lo + (uint32_t)(rng() % (L - lo + 1));
                }
                uint32_t probes = 0;
                const bool got = fx::interp_contains(at, lo, hi, c, probes);
                const bool want = std::binary_search(v.begin() + lo, v.begin() + hi, c);
                checks++;
                if (got != want) {
                    if (fails < 5) printf("MISMATCH L=%u lo=%u hi=%u c=%d got=%d want=%d\n", L, lo, hi, c, got, want);
                    fails++;
                }
                const long long over = (long long)probes - bound;
                if (over > max_over) max_over = over;
            }
        }
    };
    // empty, tiny and small runs
    for (int L = 0; L <= 40; L++)
        for (int t = 0; t < 20; t++) {
            std::vector<int32_t> v;
            for (int i = 0; i < L; i++) v.push_back((int32_t)(rng() % 200));
            run(v);
        }
    // uniform ids over a graph-sized range, clustered ids, geometric gaps, extremes
    for (int L : {64, 1000, 5000, 40000}) {
        std::vector<int32_t> u, cl, geo, ext;
        for (int i = 0; i < L; i++) u.push_back((int32_t)(rng() % 4600000));
        for (int i = 0; i < L; i++) cl.push_back((int32_t)((rng() % 8) * 100000000 + rng() % 1000));
        int64_t x = 0;
        for (int i = 0; i < L && x < 2147483647; i++) {
            x += 1 + (int64_t)(rng() % (1ull << (rng() % 24)));
            if (x < 2147483647) geo.push_back((int32_t)x);
        }
        for (int i = 0; i < L / 2; i++) { ext.push_back(i); ext.push_back(2147483647 - i); }
        run(u);
        run(cl);
        run(geo);
        run(ext);
    }
    printf("checks %lld fails %lld max_probes_over_bound %lld\n", checks, fails, max_over);
    return (fails == 0 && max_over <= 0) ? 0 : 1;
}
