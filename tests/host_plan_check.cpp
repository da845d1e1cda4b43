// Host check of the pattern compiler (csrc/pattern.cpp, compile_plan) against plain
// recomputations from the definitions: the canonical code is realised by the plan's adjacency;
// the matching order starts at canonical vertex 0 and always takes the smallest unvisited vertex
// adjacent to a visited one; backward-neighbour and same-label masks, degrees and labels per
// level; orbit representatives = smallest vertex of each orbit of the automorphism group (all
// n! orders tried); label-index slices and neighbour-label sets; tau at its closed-form special
// cases; absent labels and invalid inputs.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <set>
#include <vector>

#include "fx.h"

using namespace fx;

static int fails = 0;
#define CHECK(c)                                                              \
    do {                                                                      \
        if (!(c)) {                                                           \
            if (fails < 10) printf("FAIL line %d: %s\n", __LINE__, #c);       \
            fails++;                                                          \
        }                                                                     \
    } while (0)

static bool adjq(const Plan &P, int a, int b) { return (P.cadj[a] >> b) & 1; }

static void check_level_plan(const Plan &P, const LevelPlan &L, int first) {
    const int n = P.code_n;
    int visited = 0;
    for (int i = 0; i < n; i++) {
        const int v = L.vert[i];
        if (i == 0) {
            CHECK(v == first);
        } else {
            int want = -1;
            for (int u = 0; u < n && want < 0; u++) {
                if (visited >> u & 1) continue;
                for (int w = 0; w < n; w++)
                    if ((visited >> w & 1) && adjq(P, u, w)) { want = u; break; }
            }
            CHECK(v == want);
        }
        CHECK(L.lab[i] == P.code_lab[v]);
        int deg = 0;
        for (int w = 0; w < n; w++) deg += adjq(P, v, w);
        CHECK(L.deg[i] == deg);
        uint8_t bm = 0, im = 0;
        for (int j = 0; j < i; j++) {
            if (adjq(P, L.vert[j], v)) bm |= (uint8_t)(1 << j);
            if (P.code_lab[L.vert[j]] == P.code_lab[v]) im |= (uint8_t)(1 << j);
        }
        CHECK(L.bmask[i] == bm);
        CHECK(L.injmask[i] == im);
        visited |= 1 << v;
    }
}

int main() {
    std::mt19937_64 rng(99);
    // a data graph with 6 labels of different frequencies (label 5 absent)
    const int64_t nv = 400;
    std::vector<int32_t> lab((size_t)nv), src, dst;
    for (auto &x : lab) x = std::min<int>((int)(rng() % 5), (int)(rng() % 5));
    for (int e = 0; e < 1600; e++) { src.push_back((int32_t)(rng() % nv)); dst.push_back((int32_t)(rng() % nv)); }
    HostGraph g;
    CHECK(build_host_graph(nv, lab.data(), (int64_t)src.size(), src.data(), dst.data(), DEFAULT_SEED, 0, g) == 0);
    int checked = 0;
    for (int t = 0; t < 3000; t++) {
        const int n = 2 + (int)(rng() % 7);
        std::vector<int32_t> pl((size_t)n), pe;
        for (auto &x : pl) x = (int32_t)(rng() % 5);
        // connected: a random tree plus random extra edges
        for (int v = 1; v < n; v++) { pe.push_back((int32_t)(rng() % v)); pe.push_back(v); }
        for (int a = 0; a < n; a++)
            for (int b = a + 1; b < n; b++)
                if (rng() % 4 == 0) { pe.push_back(a); pe.push_back(b); }
        flexis_pattern fp{n, (int32_t)(pe.size() / 2), pl.data(), pe.data()};
        const int mode = (t % 2) ? FLEXIS_MODE_FULL : FLEXIS_MODE_EARLY;
        Plan P;
        CHECK(compile_plan(g, fp, 1000, 500000, 1000000, mode, P) == 0);
        CHECK(P.status == 0 && P.n == n && P.code_n == n);
        CHECK(P.want_mni == 1);
        // the code is realised by the plan's adjacency rows, labels are ranks in sorted order
        uint32_t bits = 0;
        for (int j = 1; j < n; j++)
            for (int i = 0; i < j; i++) bits = (bits << 1) | (adjq(P, i, j) ? 0u : 1u);
        CHECK(bits == P.code_bits);
        for (int i = 1; i < n; i++) CHECK(P.code_lab[i - 1] <= P.code_lab[i]);
        for (int i = 0; i < n; i++) {
            CHECK(P.lab_begin[i] == g.lab_ptr[P.code_lab[i]] && P.lab_end[i] == g.lab_ptr[P.code_lab[i] + 1]);
            uint64_t need = 0;
            for (int w = 0; w < n; w++)
                if (adjq(P, i, w)) need |= 1ull << P.code_lab[w];
            CHECK(P.need[i] == need);
        }
        CHECK(P.root_begin == P.lab_begin[0] && P.root_end == P.lab_end[0]);
        check_level_plan(P, P.greedy, 0);
        // orbits by brute force over all label- and edge-preserving permutations
        std::vector<int> orb(n);
        std::iota(orb.begin(), orb.end(), 0);
        std::vector<int> perm(n);
        std::iota(perm.begin(), perm.end(), 0);
        do {
            bool ok = true;
            for (int a = 0; a < n && ok; a++) {
                if (P.code_lab[a] != P.code_lab[perm[a]]) ok = false;
                for (int b = 0; b < n && ok; b++)
                    if (adjq(P, a, b) != adjq(P, perm[a], perm[b])) ok = false;
            }
            if (ok)
                for (int a = 0; a < n; a++) orb[perm[a]] = std::min(orb[perm[a]], orb[a]);
        } while (std::next_permutation(perm.begin(), perm.end()));
        // orb[a] is the smallest vertex mapped to a by some automorphism (the group is closed
        // under inverses, so that is the smallest vertex of a's orbit)
        std::vector<int> reps;
        for (int a = 0; a < n; a++)
            if (orb[a] == a) reps.push_back(a);
        CHECK(P.n_orb == (int)reps.size());
        for (int k = 0; k < P.n_orb && k < (int)reps.size(); k++) check_level_plan(P, P.orb[k], reps[(size_t)k]);
        // tau and the cap
        CHECK(P.tau == (1000 * ((int64_t)(n - 1) * 500000 + 1000000)) / ((int64_t)n * 1000000));
        CHECK(P.cap == (mode == FLEXIS_MODE_EARLY ? std::max<int64_t>(P.tau, 1) : CAP_INF));
        checked++;
    }
    // tau at its special cases: lambda = 1 -> sigma, lambda = 0 -> floor(sigma / n), exact rounding
    for (int n = 2; n <= 8; n++)
        for (int64_t s : {1, 2, 3, 7, 1000, 20000}) {
            CHECK(tau_exact(s, 1, 1, n) == s);
            CHECK(tau_exact(s, 0, 1, n) == s / n);
        }
    CHECK(tau_exact(3, 600000, 1000000, 6) == 2);
    CHECK(tau_exact(2, 1, 4, 3) == 1);
    // absent label, invalid inputs
    {
        int32_t l2[2] = {0, 5}, e2[2] = {0, 1};
        flexis_pattern fp{2, 1, l2, e2};
        Plan P;
        CHECK(compile_plan(g, fp, 10, 1, 2, FLEXIS_MODE_EARLY, P) == 0);
        CHECK((P.flags & FLEXIS_FLAG_ABSENT_LABEL) && P.root_begin == P.root_end);
        int32_t l3[3] = {0, 1, 2}, e3[2] = {0, 1};
        flexis_pattern disc{3, 1, l3, e3};
        CHECK(compile_plan(g, disc, 10, 1, 2, FLEXIS_MODE_EARLY, P) == FLEXIS_E_INVALID);
        flexis_pattern one{1, 0, l3, e3};
        CHECK(compile_plan(g, one, 10, 1, 2, FLEXIS_MODE_EARLY, P) == FLEXIS_E_INVALID);
        CHECK(compile_plan(g, fp, 0, 1, 2, FLEXIS_MODE_EARLY, P) == FLEXIS_E_INVALID);
        CHECK(compile_plan(g, fp, 10, 3, 2, FLEXIS_MODE_EARLY, P) == FLEXIS_E_INVALID);
        int32_t self[2] = {0, 0};
        flexis_pattern loop{2, 1, l2, self};
        CHECK(compile_plan(g, loop, 10, 1, 2, FLEXIS_MODE_EARLY, P) == FLEXIS_E_INVALID);
        // no MNI: no orbit plans
        int32_t l4[2] = {0, 1};
        flexis_pattern ok{2, 1, l4, e2};
        CHECK(compile_plan(g, ok, 10, 1, 2, FLEXIS_MODE_EARLY | FLEXIS_MODE_NO_MNI, P) == 0);
        CHECK(P.want_mni == 0 && P.n_orb == 0 && (P.flags & FLEXIS_FLAG_MNI_SKIPPED));
    }
    printf("plans %d fails %d\n", checked, fails);
    return fails == 0 ? 0 : 1;
}
