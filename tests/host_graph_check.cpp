// Host check of the data-graph build (csrc/graph.cpp, build_host_graph) against a plain
// recomputation: label ranks by ascending frequency (ties by id), deduplicated adjacency sorted
// by (rank, id), per-vertex label runs and their degree sentinel, vertex records, the
// label-partitioned root index in (H(seed, v), v) order or vertex-id order, label pairs on edges,
// and the counters of dropped self-loops and repeated edges; for directed graphs the out-, in-
// and mutual-neighbour lists with their records.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <map>
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

static void check_graph(int64_t nv, const std::vector<int32_t> &lab, const std::vector<int32_t> &src,
                        const std::vector<int32_t> &dst, uint64_t seed, int id_order) {
    HostGraph g;
    const int rc = build_host_graph(nv, lab.data(), (int64_t)src.size(), src.data(), dst.data(), seed, id_order, g);
    CHECK(rc == 0);
    if (rc) return;
    // ranks
    std::map<int32_t, int64_t> cnt;
    for (int64_t v = 0; v < nv; v++) cnt[lab[(size_t)v]]++;
    std::vector<std::pair<int64_t, int32_t>> order;
    for (auto &kv : cnt) order.push_back({kv.second, kv.first});
    std::sort(order.begin(), order.end());
    std::map<int32_t, int32_t> rank;
    for (size_t r = 0; r < order.size(); r++) rank[order[r].second] = (int32_t)r;
    CHECK(g.nl == (int32_t)order.size());
    for (auto &kv : rank) {
        CHECK(g.rank_of[(size_t)kv.first] == kv.second);
        CHECK(g.label_of_rank[(size_t)kv.second] == kv.first);
    }
    // neighbour sets, dropped edges
    std::vector<std::set<int32_t>> N((size_t)nv);
    std::set<std::pair<int32_t, int32_t>> und;
    int64_t loops = 0, kept_edges = 0;
    for (size_t e = 0; e < src.size(); e++) {
        const int32_t a = src[e], b = dst[e];
        if (a == b) { loops++; continue; }
        kept_edges++;
        und.insert({std::min(a, b), std::max(a, b)});
        N[(size_t)a].insert(b);
        N[(size_t)b].insert(a);
    }
    CHECK(g.self_loops == loops);
    CHECK(g.duplicates == kept_edges - (int64_t)und.size());
    CHECK(g.n_arcs == 2 * (int64_t)und.size());
    int32_t maxdeg = 0;
    for (int64_t v = 0; v < nv; v++) {
        const auto &nb = N[(size_t)v];
        std::vector<std::pair<int32_t, int32_t>> want;
        for (int32_t w : nb) want.push_back({rank[lab[(size_t)w]], w});
        std::sort(want.begin(), want.end());
        const VRec &r = g.vrec[(size_t)v];
        maxdeg = std::max<int32_t>(maxdeg, (int32_t)want.size());
        CHECK(r.deg == (uint32_t)want.size());
        uint64_t mask = 0;
        uint32_t nrun = 0;
        for (size_t t = 0; t < want.size(); t++) {
            CHECK(g.adj[r.adj + t] == want[t].second);
            if (want[t].first < 64) mask |= 1ull << want[t].first;
            if (t == 0 || want[t].first != want[t - 1].first) {
                CHECK(g.runs[r.run + nrun] == (((uint32_t)want[t].first << 24) | (uint32_t)t));
                nrun++;
            }
        }
        CHECK(g.runs[r.run + nrun] == ((RUN_SENTINEL_LABEL << 24) | (uint32_t)want.size()));
        CHECK(r.meta == ((nrun << 8) | (uint32_t)rank[lab[(size_t)v]]));
        CHECK(r.nbr_labels == mask);
    }
    CHECK(g.max_degree == maxdeg);
    // root index
    for (int32_t q = 0; q < g.nl; q++) {
        std::vector<std::pair<uint64_t, int32_t>> want;
        for (int64_t v = 0; v < nv; v++)
            if (rank[lab[(size_t)v]] == q) want.push_back({id_order ? 0 : root_hash(seed, v), (int32_t)v});
        std::sort(want.begin(), want.end());
        CHECK(g.lab_ptr[(size_t)q + 1] - g.lab_ptr[(size_t)q] == (int32_t)want.size());
        for (size_t i = 0; i < want.size(); i++) CHECK(g.lab_vtx[(size_t)g.lab_ptr[(size_t)q] + i] == want[i].second);
    }
    // rank pairs on data edges
    std::set<std::pair<int32_t, int32_t>> pairs;
    for (auto &e : und) {
        const int32_t a = rank[lab[(size_t)e.first]], b = rank[lab[(size_t)e.second]];
        pairs.insert({std::min(a, b), std::max(a, b)});
    }
    std::set<std::pair<int32_t, int32_t>> got(g.label_pairs.begin(), g.label_pairs.end());
    CHECK(got == pairs);
}

// Directed build: for every vertex the out-, in- and mutual-neighbour lists (each sorted by
// (rank, id) with its label runs and sentinel) and their records; the out record carries the
// one-hop filter data of the union (distinct neighbours either way, their labels).
static void check_directed(int64_t nv, const std::vector<int32_t> &lab, const std::vector<int32_t> &src,
                           const std::vector<int32_t> &dst) {
    HostGraph g;
    const int rc = build_host_graph(nv, lab.data(), (int64_t)src.size(), src.data(), dst.data(), 0x5EEDull, 0, g, 1);
    CHECK(rc == 0);
    if (rc) return;
    CHECK(g.directed == 1 && (int64_t)g.vrec.size() == std::max<int64_t>(3 * nv, 1));
    std::map<int32_t, int64_t> cnt;
    for (int64_t v = 0; v < nv; v++) cnt[lab[(size_t)v]]++;
    std::vector<std::pair<int64_t, int32_t>> order;
    for (auto &kv : cnt) order.push_back({kv.second, kv.first});
    std::sort(order.begin(), order.end());
    std::map<int32_t, int32_t> rank;
    for (size_t r = 0; r < order.size(); r++) rank[order[r].second] = (int32_t)r;
    std::vector<std::set<int32_t>> out((size_t)nv), in((size_t)nv);
    std::set<std::pair<int32_t, int32_t>> arcs;
    int64_t loops = 0;
    for (size_t e = 0; e < src.size(); e++) {
        if (src[e] == dst[e]) { loops++; continue; }
        arcs.insert({src[e], dst[e]});
        out[(size_t)src[e]].insert(dst[e]);
        in[(size_t)dst[e]].insert(src[e]);
    }
    CHECK(g.self_loops == loops);
    CHECK(g.n_arcs == (int64_t)arcs.size());
    CHECK(g.duplicates == (int64_t)src.size() - loops - (int64_t)arcs.size());
    int32_t maxdeg = 0;
    for (int64_t v = 0; v < nv; v++) {
        std::set<int32_t> mut, uni;
        for (int32_t w : out[(size_t)v]) {
            uni.insert(w);
            if (in[(size_t)v].count(w)) mut.insert(w);
        }
        for (int32_t w : in[(size_t)v]) uni.insert(w);
        const std::set<int32_t> *lists[3] = {&out[(size_t)v], &in[(size_t)v], &mut};
        for (int k = 0; k < 3; k++) {
            std::vector<std::pair<int32_t, int32_t>> want;
            for (int32_t w : *lists[k]) want.push_back({rank[lab[(size_t)w]], w});
            std::sort(want.begin(), want.end());
            const VRec &r = g.vrec[(size_t)(k * nv + v)];
            uint32_t nrun = 0;
            uint64_t mask = 0;
            for (size_t t = 0; t < want.size(); t++) {
                CHECK(g.adj[r.adj + t] == want[t].second);
                if (want[t].first < 64) mask |= 1ull << want[t].first;
                if (t == 0 || want[t].first != want[t - 1].first) {
                    CHECK(g.runs[r.run + nrun] == (((uint32_t)want[t].first << 24) | (uint32_t)t));
                    nrun++;
                }
            }
            CHECK(g.runs[r.run + nrun] == ((RUN_SENTINEL_LABEL << 24) | (uint32_t)want.size()));
            CHECK(r.meta == ((nrun << 8) | (uint32_t)rank[lab[(size_t)v]]));
            if (k > 0) {
                CHECK(r.deg == (uint32_t)want.size());
                CHECK(r.nbr_labels == mask);
            }
        }
        uint64_t umask = 0;
        for (int32_t w : uni)
            if (rank[lab[(size_t)w]] < 64) umask |= 1ull << rank[lab[(size_t)w]];
        CHECK(g.vrec[(size_t)v].deg == (uint32_t)uni.size());
        CHECK(g.vrec[(size_t)v].nbr_labels == umask);
        maxdeg = std::max<int32_t>(maxdeg, (int32_t)uni.size());
    }
    CHECK(g.max_degree == maxdeg);
}

int main() {
    std::mt19937_64 rng(2024);
    int graphs = 0;
    for (int64_t nv : {1, 2, 7, 60, 700, 5000})
        for (int L : {1, 3, 20, 70})
            for (int rep = 0; rep < 3; rep++) {
                std::vector<int32_t> lab((size_t)nv), src, dst;
                for (auto &x : lab) {
                    // skewed label ids, some ids absent
                    const int a = (int)(rng() % L), b = (int)(rng() % L);
                    x = std::min(a, b) * 2;
                }
                const int64_t ne = nv * (1 + (int64_t)(rng() % 6));
                for (int64_t e = 0; e < ne; e++) {
                    int32_t a = (int32_t)(rng() % nv), b = (int32_t)(rng() % nv);
                    if (rng() % 10 == 0) b = a;                           // self-loop
                    src.push_back(a);
                    dst.push_back(b);
                    if (rng() % 8 == 0) { src.push_back(b); dst.push_back(a); }  // repeat
                }
                // a hub
                for (int64_t v = 1; v < nv && v < 400; v++) { src.push_back(0); dst.push_back((int32_t)v); }
                for (int id_order : {0, 1}) {
                    check_graph(nv, lab, src, dst, 0x5EEDull + (uint64_t)rep, id_order);
                    graphs++;
                }
                check_directed(nv, lab, src, dst);
                graphs++;
            }
    printf("graphs %d fails %d\n", graphs, fails);
    return fails == 0 ? 0 : 1;
}
