// Host-side construction of the resident data-graph layout (done once per graph).
//
// The paper's data graph is a single large vertex-labelled graph (Sec. 2.2) read by an
// undirected loader (Sec. 4.1).  Layout built here and mirrored on the device:
//   adj      : per vertex, neighbours sorted by (label rank, id)  -> label slices are contiguous
//   runs     : per vertex, one 32-bit entry per label present among its neighbours
//              (rank << 24 | offset of the slice within the row), then a sentinel
//              (0xFF << 24 | degree), so a slice is [entry_j, entry_{j+1}) in one warp load
//   vrec     : per vertex {row offset, run offset, run count, rank label} (one 16-byte load)
//   lab_vtx  : vertices grouped by label rank; inside a group in greedy-root order
//              (H(seed, v), v) so a pattern's roots are one contiguous, pre-ordered slice
#include <algorithm>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

#include "fx.h"

namespace fx {

uint64_t root_hash(uint64_t seed, int64_t r) {
    // one SplitMix64 step (Steele, Lea, Flood 2014) from state seed XOR r
    uint64_t z = (seed ^ (uint64_t)r) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class F>
static void parallel_for(int64_t n, F f) {
    int T = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < 100000) T = 1;
    std::vector<std::thread> th;
    int64_t chunk = (n + T - 1) / T;
    for (int t = 0; t < T; t++) {
        int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
        if (lo >= hi) break;
        th.emplace_back([=] { f(lo, hi); });
    }
    for (auto &x : th) x.join();
}

static void finish_index(HostGraph &g, const std::vector<uint8_t> &rk, int64_t nv, uint64_t seed, int id_order);

// Per-vertex neighbour rows (CSR off/nbr) sorted by (rank, id) without repeats, written as one
// list kind of the layout: adjacency at adj_base, label runs + sentinel at run_base, one VRec
// per vertex into rec[0, nv).  lists_bytes: adjacency entries and run entries of each vertex.
struct Rows {
    std::vector<int64_t> off;  // [nv + 1]
    std::vector<int32_t> nbr;
};

static Rows sorted_rows(int64_t nv, const std::vector<int64_t> &deg, const std::vector<int32_t> &rk,
                        const std::function<void(std::vector<int64_t> &, std::vector<int32_t> &)> &fill) {
    Rows r;
    r.off.assign((size_t)nv + 1, 0);
    for (int64_t v = 0; v < nv; v++) r.off[(size_t)v + 1] = r.off[(size_t)v] + deg[(size_t)v];
    std::vector<int32_t> tmp((size_t)std::max<int64_t>(r.off[(size_t)nv], 1));
    std::vector<int64_t> pos(r.off.begin(), r.off.end() - 1);
    fill(pos, tmp);
    std::vector<int64_t> kept((size_t)nv, 0);
    parallel_for(nv, [&](int64_t lo, int64_t hi) {
        std::vector<uint64_t> key;
        for (int64_t v = lo; v < hi; v++) {
            const int64_t a = r.off[(size_t)v], b = r.off[(size_t)v + 1];
            key.resize((size_t)(b - a));
            for (int64_t t = a; t < b; t++) {
                const int32_t w = tmp[(size_t)t];
                key[(size_t)(t - a)] = ((uint64_t)(uint32_t)rk[(size_t)w] << 32) | (uint32_t)w;
            }
            std::sort(key.begin(), key.end());
            const size_t k = (size_t)(std::unique(key.begin(), key.end()) - key.begin());
            for (size_t t = 0; t < k; t++) tmp[(size_t)a + t] = (int32_t)(key[t] & 0xFFFFFFFFu);
            kept[(size_t)v] = (int64_t)k;
        }
    });
    std::vector<int64_t> off2((size_t)nv + 1, 0);
    for (int64_t v = 0; v < nv; v++) off2[(size_t)v + 1] = off2[(size_t)v] + kept[(size_t)v];
    r.nbr.resize((size_t)std::max<int64_t>(off2[(size_t)nv], 1));
    parallel_for(nv, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; v++)
            std::copy(tmp.begin() + r.off[(size_t)v], tmp.begin() + r.off[(size_t)v] + kept[(size_t)v],
                      r.nbr.begin() + off2[(size_t)v]);
    });
    r.off.swap(off2);
    return r;
}

// Directed data graph: arcs as given.  Each vertex has three rows -- out-neighbours, in-neighbours
// and mutual neighbours (both arcs) -- laid out one after the other in `adj` and `runs`, with one
// VRec array per row kind (vrec[k * nv + v]).  The out record carries the vertex's one-hop filter
// data for the union of its neighbours (degree |out u in|, neighbour labels).
static int build_directed(int64_t nv, int64_t ne, const int32_t *src, const int32_t *dst,
                          const std::vector<int32_t> &rk, HostGraph &g) {
    std::vector<int64_t> dout((size_t)nv + 1, 0), din((size_t)nv + 1, 0);
    for (int64_t e = 0; e < ne; e++) {
        if (src[e] == dst[e]) { g.self_loops++; continue; }
        dout[(size_t)src[e]]++;
        din[(size_t)dst[e]]++;
    }
    Rows out = sorted_rows(nv, dout, rk, [&](std::vector<int64_t> &pos, std::vector<int32_t> &tmp) {
        for (int64_t e = 0; e < ne; e++)
            if (src[e] != dst[e]) tmp[(size_t)pos[(size_t)src[e]]++] = dst[e];
    });
    Rows in = sorted_rows(nv, din, rk, [&](std::vector<int64_t> &pos, std::vector<int32_t> &tmp) {
        for (int64_t e = 0; e < ne; e++)
            if (src[e] != dst[e]) tmp[(size_t)pos[(size_t)dst[e]]++] = src[e];
    });
    // mutual = out n in, rows merged in (rank, id) order
    std::vector<int64_t> dmut((size_t)nv + 1, 0);
    for (int64_t v = 0; v < nv; v++) {
        int64_t a = out.off[(size_t)v], ae = out.off[(size_t)v + 1], b = in.off[(size_t)v], be = in.off[(size_t)v + 1];
        while (a < ae && b < be) {
            const uint64_t x = ((uint64_t)(uint32_t)rk[(size_t)out.nbr[(size_t)a]] << 32) | (uint32_t)out.nbr[(size_t)a];
            const uint64_t y = ((uint64_t)(uint32_t)rk[(size_t)in.nbr[(size_t)b]] << 32) | (uint32_t)in.nbr[(size_t)b];
            if (x == y) { dmut[(size_t)v]++; a++; b++; } else if (x < y) a++; else b++;
        }
    }
    Rows mut = sorted_rows(nv, dmut, rk, [&](std::vector<int64_t> &pos, std::vector<int32_t> &tmp) {
        for (int64_t v = 0; v < nv; v++) {
            int64_t a = out.off[(size_t)v], ae = out.off[(size_t)v + 1], b = in.off[(size_t)v], be = in.off[(size_t)v + 1];
            while (a < ae && b < be) {
                const int32_t wa = out.nbr[(size_t)a], wb = in.nbr[(size_t)b];
                const uint64_t x = ((uint64_t)(uint32_t)rk[(size_t)wa] << 32) | (uint32_t)wa;
                const uint64_t y = ((uint64_t)(uint32_t)rk[(size_t)wb] << 32) | (uint32_t)wb;
                if (x == y) { tmp[(size_t)pos[(size_t)v]++] = wa; a++; b++; } else if (x < y) a++; else b++;
            }
        }
    });
    const Rows *kinds[3] = {&out, &in, &mut};
    int64_t arcs = 0, nruns = 0;
    std::vector<int64_t> koff((size_t)3 * nv), roff((size_t)3 * nv);
    std::vector<int32_t> nrun((size_t)3 * nv);
    for (int64_t v = 0; v < nv; v++)
        for (int k = 0; k < 3; k++) {
            const Rows &R = *kinds[k];
            int32_t r = 0;
            for (int64_t t = R.off[(size_t)v]; t < R.off[(size_t)v + 1]; t++)
                if (t == R.off[(size_t)v] || rk[(size_t)R.nbr[(size_t)t]] != rk[(size_t)R.nbr[(size_t)t - 1]]) r++;
            koff[(size_t)(k * nv + v)] = arcs;
            roff[(size_t)(k * nv + v)] = nruns;
            nrun[(size_t)(k * nv + v)] = r;
            arcs += R.off[(size_t)v + 1] - R.off[(size_t)v];
            nruns += r + 1;
        }
    if (arcs >= (int64_t)UINT32_MAX || nruns >= (int64_t)UINT32_MAX) return FLEXIS_E_UNSUPPORTED;
    g.n_arcs = out.off[(size_t)nv];
    g.duplicates = (ne - g.self_loops) - g.n_arcs;
    g.adj.resize((size_t)std::max<int64_t>(arcs, 1));
    g.runs.resize((size_t)std::max<int64_t>(nruns, 1));
    g.vrec.resize((size_t)std::max<int64_t>(3 * nv, 1));
    for (int64_t v = 0; v < nv; v++) {
        uint64_t union_labels = 0;
        for (int k = 0; k < 3; k++) {
            const Rows &R = *kinds[k];
            const int64_t a = R.off[(size_t)v], len = R.off[(size_t)v + 1] - a;
            const int64_t o = koff[(size_t)(k * nv + v)], ro = roff[(size_t)(k * nv + v)];
            int64_t j = 0;
            uint64_t lm = 0;
            for (int64_t t = 0; t < len; t++) {
                const int32_t w = R.nbr[(size_t)(a + t)];
                g.adj[(size_t)(o + t)] = w;
                if (rk[(size_t)w] < 64) lm |= 1ull << rk[(size_t)w];
                if (t == 0 || rk[(size_t)w] != rk[(size_t)R.nbr[(size_t)(a + t - 1)]])
                    g.runs[(size_t)(ro + j++)] = ((uint32_t)rk[(size_t)w] << 24) | (uint32_t)t;
            }
            g.runs[(size_t)(ro + j)] = (RUN_SENTINEL_LABEL << 24) | (uint32_t)len;
            union_labels |= lm;
            if (len >= (1 << 24)) return FLEXIS_E_UNSUPPORTED;
            g.vrec[(size_t)(k * nv + v)] = VRec{(uint32_t)o, (uint32_t)ro, (uint32_t)len,
                                               ((uint32_t)j << 8) | (uint32_t)rk[(size_t)v], lm, 0};
        }
        const int64_t udeg = (out.off[(size_t)v + 1] - out.off[(size_t)v]) + (in.off[(size_t)v + 1] - in.off[(size_t)v]) -
                             (mut.off[(size_t)v + 1] - mut.off[(size_t)v]);
        if (udeg >= (1 << 24)) return FLEXIS_E_UNSUPPORTED;
        g.vrec[(size_t)v].deg = (uint32_t)udeg;  // the filter: distinct neighbours either way
        g.vrec[(size_t)v].nbr_labels = union_labels;
        g.max_degree = std::max<int32_t>(g.max_degree, (int32_t)udeg);
    }
    return FLEXIS_OK;
}

int label_ranks(int64_t nv, const int32_t *labels, HostGraph &g, std::vector<uint8_t> &rk) {
    int32_t nl_ids = 0;
    for (int64_t v = 0; v < nv; v++) {
        if (labels[v] < 0) return FLEXIS_E_INVALID;
        nl_ids = std::max(nl_ids, labels[v] + 1);
    }
    g.nl_ids = nl_ids;
    // label ranks: ascending frequency, ties by id
    std::vector<int64_t> cnt((size_t)nl_ids, 0);
    for (int64_t v = 0; v < nv; v++) cnt[(size_t)labels[v]]++;
    std::vector<int32_t> present;
    for (int32_t a = 0; a < nl_ids; a++)
        if (cnt[(size_t)a] > 0) present.push_back(a);
    std::sort(present.begin(), present.end(), [&](int32_t a, int32_t b) {
        return cnt[(size_t)a] != cnt[(size_t)b] ? cnt[(size_t)a] < cnt[(size_t)b] : a < b;
    });
    if (present.size() >= RUN_SENTINEL_LABEL) return FLEXIS_E_UNSUPPORTED;
    g.nl = (int32_t)present.size();
    g.rank_of.assign((size_t)nl_ids, -1);
    g.label_of_rank = present;
    g.lab_ptr.assign((size_t)g.nl + 1, 0);
    for (size_t r = 0; r < present.size(); r++) {
        g.rank_of[(size_t)present[r]] = (int32_t)r;
        g.lab_ptr[r + 1] = g.lab_ptr[r] + (int32_t)cnt[(size_t)present[r]];
    }
    rk.assign((size_t)std::max<int64_t>(nv, 1), 0);
    for (int64_t v = 0; v < nv; v++) rk[(size_t)v] = (uint8_t)g.rank_of[(size_t)labels[v]];
    return FLEXIS_OK;
}

int build_host_graph(int64_t nv, const int32_t *labels, int64_t ne, const int32_t *src,
                     const int32_t *dst, uint64_t seed, int id_order, HostGraph &g, int directed) {
    if (nv < 0 || ne < 0 || (nv > 0 && !labels) || (ne > 0 && (!src || !dst)))
        return FLEXIS_E_INVALID;
    if (nv >= (int64_t)INT32_MAX) return FLEXIS_E_UNSUPPORTED;
    g = HostGraph();
    g.nv = nv;
    g.seed = seed;
    for (int64_t v = 0; v < nv; v++)
        if (labels[v] < 0) return FLEXIS_E_INVALID;
    for (int64_t e = 0; e < ne; e++)
        if (src[e] < 0 || dst[e] < 0 || src[e] >= nv || dst[e] >= nv) return FLEXIS_E_INVALID;
    std::vector<uint8_t> rk;
    const int lrc = label_ranks(nv, labels, g, rk);
    if (lrc) return lrc;
    g.directed = directed ? 1 : 0;
    if (directed) {
        std::vector<int32_t> rk32(rk.begin(), rk.end());
        const int rc = build_directed(nv, ne, src, dst, rk32, g);
        if (rc) return rc;
        finish_index(g, rk, nv, seed, id_order);
        return FLEXIS_OK;
    }

    // arcs in both directions
    std::vector<int64_t> deg((size_t)nv + 1, 0);
    for (int64_t e = 0; e < ne; e++) {
        if (src[e] == dst[e]) { g.self_loops++; continue; }
        deg[(size_t)src[e]]++;
        deg[(size_t)dst[e]]++;
    }
    std::vector<int64_t> off((size_t)nv + 1, 0);
    for (int64_t v = 0; v < nv; v++) off[(size_t)v + 1] = off[(size_t)v] + deg[(size_t)v];
    if (off[(size_t)nv] >= (int64_t)UINT32_MAX) return FLEXIS_E_UNSUPPORTED;
    std::vector<int32_t> tmp((size_t)std::max<int64_t>(off[(size_t)nv], 1));
    {
        std::vector<int64_t> fill(off.begin(), off.end() - 1);
        for (int64_t e = 0; e < ne; e++) {
            if (src[e] == dst[e]) continue;
            tmp[(size_t)fill[(size_t)src[e]]++] = dst[e];
            tmp[(size_t)fill[(size_t)dst[e]]++] = src[e];
        }
    }
    // sort each row by (rank, id), drop repeats
    std::vector<int64_t> kept((size_t)nv, 0);
    parallel_for(nv, [&](int64_t lo, int64_t hi) {
        std::vector<uint64_t> key;
        for (int64_t v = lo; v < hi; v++) {
            int64_t a = off[(size_t)v], b = off[(size_t)v + 1];
            key.resize((size_t)(b - a));
            for (int64_t t = a; t < b; t++) {
                int32_t w = tmp[(size_t)t];
                key[(size_t)(t - a)] = ((uint64_t)rk[(size_t)w] << 32) | (uint32_t)w;
            }
            std::sort(key.begin(), key.end());
            size_t k = (size_t)(std::unique(key.begin(), key.end()) - key.begin());
            for (size_t t = 0; t < k; t++) tmp[(size_t)a + t] = (int32_t)(key[t] & 0xFFFFFFFFu);
            kept[(size_t)v] = (int64_t)k;
        }
    });
    int64_t arcs = 0;
    int64_t nruns = 0;
    std::vector<int64_t> koff((size_t)nv + 1, 0), roff((size_t)nv + 1, 0);
    std::vector<int32_t> nrun((size_t)nv, 0);
    parallel_for(nv, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; v++) {
            int64_t a = off[(size_t)v];
            int32_t r = 0;
            for (int64_t t = 0; t < kept[(size_t)v]; t++)
                if (t == 0 || rk[(size_t)tmp[(size_t)(a + t)]] != rk[(size_t)tmp[(size_t)(a + t - 1)]]) r++;
            nrun[(size_t)v] = r;
        }
    });
    for (int64_t v = 0; v < nv; v++) {
        koff[(size_t)v] = arcs;
        roff[(size_t)v] = nruns;
        arcs += kept[(size_t)v];
        nruns += nrun[(size_t)v] + 1;
        g.max_degree = std::max<int32_t>(g.max_degree, (int32_t)kept[(size_t)v]);
    }
    if (arcs >= (int64_t)UINT32_MAX || nruns >= (int64_t)UINT32_MAX) return FLEXIS_E_UNSUPPORTED;
    if (g.max_degree >= (1 << 24)) return FLEXIS_E_UNSUPPORTED;
    g.duplicates = (off[(size_t)nv] - arcs) / 2;
    g.n_arcs = arcs;
    g.adj.resize((size_t)std::max<int64_t>(arcs, 1));
    g.runs.resize((size_t)std::max<int64_t>(nruns, 1));
    g.vrec.resize((size_t)std::max<int64_t>(nv, 1));
    parallel_for(nv, [&](int64_t lo, int64_t hi) {
        for (int64_t v = lo; v < hi; v++) {
            int64_t a = off[(size_t)v], k = kept[(size_t)v];
            int64_t o = koff[(size_t)v], ro = roff[(size_t)v];
            int64_t j = 0;
            uint64_t lm = 0;
            for (int64_t t = 0; t < k; t++) {
                int32_t w = tmp[(size_t)(a + t)];
                g.adj[(size_t)(o + t)] = w;
                if (rk[(size_t)w] < 64) lm |= 1ull << rk[(size_t)w];
                if (t == 0 || rk[(size_t)w] != rk[(size_t)tmp[(size_t)(a + t - 1)]])
                    g.runs[(size_t)(ro + j++)] = ((uint32_t)rk[(size_t)w] << 24) | (uint32_t)t;
            }
            g.runs[(size_t)(ro + j)] = (RUN_SENTINEL_LABEL << 24) | (uint32_t)k;
            g.vrec[(size_t)v] = VRec{(uint32_t)o, (uint32_t)ro, (uint32_t)k,
                                     ((uint32_t)j << 8) | (uint32_t)rk[(size_t)v], lm, 0};
        }
    });
    finish_index(g, rk, nv, seed, id_order);
    // label pairs present on data edges (level-2 candidates of Algorithm 1)
    std::vector<uint8_t> pair((size_t)g.nl * (size_t)std::max(g.nl, 1), 0);
    for (int64_t v = 0; v < nv; v++)
        for (int64_t t = koff[(size_t)v]; t < koff[(size_t)v] + kept[(size_t)v]; t++) {
            int a = rk[(size_t)v], b = rk[(size_t)g.adj[(size_t)t]];
            if (a <= b) pair[(size_t)a * (size_t)g.nl + (size_t)b] = 1;
        }
    for (int a = 0; a < g.nl; a++)
        for (int b = a; b < g.nl; b++)
            if (pair[(size_t)a * (size_t)g.nl + (size_t)b]) g.label_pairs.emplace_back(a, b);
    return FLEXIS_OK;
}

// Label-partitioned vertex index in greedy-root order.
static void finish_index(HostGraph &g, const std::vector<uint8_t> &rk, int64_t nv, uint64_t seed, int id_order) {
    g.lab_ptr.assign((size_t)g.nl + 1, 0);
    for (int64_t v = 0; v < nv; v++) g.lab_ptr[(size_t)rk[(size_t)v] + 1]++;
    for (int32_t r = 0; r < g.nl; r++) g.lab_ptr[(size_t)r + 1] += g.lab_ptr[(size_t)r];
    std::vector<uint64_t> hv((size_t)std::max<int64_t>(nv, 1));
    parallel_for(nv, [&](int64_t lo, int64_t hi) {
        // root-order variant: by vertex id (the hash key dropped)
        for (int64_t v = lo; v < hi; v++) hv[(size_t)v] = id_order ? 0 : root_hash(seed, v);
    });
    g.lab_vtx.resize((size_t)std::max<int64_t>(nv, 1));
    {
        std::vector<int32_t> fill(g.lab_ptr.begin(), g.lab_ptr.end() - 1);
        for (int64_t v = 0; v < nv; v++) g.lab_vtx[(size_t)fill[rk[(size_t)v]]++] = (int32_t)v;
    }
    for (int32_t r = 0; r < g.nl; r++) {
        auto b = g.lab_vtx.begin() + g.lab_ptr[(size_t)r], e = g.lab_vtx.begin() + g.lab_ptr[(size_t)r + 1];
        std::sort(b, e, [&](int32_t x, int32_t y) {
            return hv[(size_t)x] != hv[(size_t)y] ? hv[(size_t)x] < hv[(size_t)y] : x < y;
        });
    }
}

}  // namespace fx
