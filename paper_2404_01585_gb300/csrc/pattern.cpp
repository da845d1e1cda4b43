// Host pattern compiler: canonical form (the role Bliss plays in the paper, Sec. 2.1.5),
// automorphism orbits, matching orders, tau (Eq. tau), and candidate generation by core-group
// merging (Algorithms 2-4, Sec. 3.2.1).
#include <algorithm>
#include <array>
#include <atomic>
#include <cstring>
#include <functional>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "fx.h"

namespace fx {

bool Code::operator<(const Code &o) const {
    if (n != o.n) return n < o.n;
    for (int i = 0; i < n; i++)
        if (lab[i] != o.lab[i]) return lab[i] < o.lab[i];
    return bits < o.bits;
}

bool Code::operator==(const Code &o) const {
    if (n != o.n || bits != o.bits) return false;
    for (int i = 0; i < n; i++)
        if (lab[i] != o.lab[i]) return false;
    return true;
}

size_t CodeHash::operator()(const Code &c) const {
    uint64_t h = 0x9E3779B97F4A7C15ull * (uint64_t)(c.n + 1) ^ c.bits;
    for (int i = 0; i < c.n; i++) h = (h ^ (uint64_t)(uint32_t)c.lab[i]) * 0x100000001B3ull;
    return (size_t)(h ^ (h >> 29));
}

static inline bool has(const Pat &p, int i, int j) { return (p.adj[i] >> j) & 1; }

bool connected(const Pat &p) {
    if (p.n == 0) return false;
    int seen = 1, frontier = 1;
    while (frontier) {
        int nxt = 0;
        for (int u = 0; u < p.n; u++)
            if (frontier >> u & 1) nxt |= p.adj[u];
        nxt &= ~seen;
        seen |= nxt;
        frontier = nxt;
    }
    return seen == (1 << p.n) - 1;
}

int edge_count(const Pat &p) {
    int m = 0;
    for (int i = 0; i < p.n; i++) m += __builtin_popcount(p.adj[i]);
    return m / 2;
}

// ---------------------------------------------------------------- canonical form
// Code of an order (position -> vertex): labels in order, then for columns j = 1..n-1 and rows
// i = 0..j-1 the bit "not adjacent"; the canonical code is the lexicographic minimum over all
// orders.  Search: positions are filled left to right; the label of each position is forced
// (sorted label multiset), and a partial order whose bit prefix already exceeds the best
// prefix is pruned.  Twins -- two vertices of one label with the same neighbours apart from
// each other -- are exchanged by an automorphism that fixes every other vertex, so at each
// position only the lowest-numbered unused vertex of a set of twins is tried: the orders skipped
// are images of tried ones under that automorphism and give the same codes.  The minimum over
// the pruned search equals the minimum over all n! orders.
namespace {
struct CanonSearch {
    const Pat *p;
    int n;
    int32_t slab[MAXN];
    int perm[MAXN];
    int best_perm[MAXN];
    uint32_t best_bits;
    bool have;
    int total_bits;
    uint32_t twin_below[MAXN];  // lower-numbered twins of each vertex

    void rec(int pos, int used, uint32_t bits, int nb) {
        if (pos == n) {
            if (!have || bits < best_bits) {
                best_bits = bits;
                memcpy(best_perm, perm, sizeof(int) * n);
                have = true;
            }
            return;
        }
        if (pos >= MAXN) return;
        for (int w = 0; w < n; w++) {
            if (used >> w & 1) continue;
            if (p->lab[w] != slab[pos]) continue;
            if (twin_below[w] & ~(uint32_t)used) continue;  // an unused lower twin stands for w
            uint32_t b = bits;
            for (int i = 0; i < pos; i++) b = (b << 1) | (has(*p, perm[i], w) ? 0u : 1u);
            int nb2 = nb + pos;
            // prune: this prefix already exceeds the best code's prefix
            if (have && nb2 > 0 && b > (best_bits >> (total_bits - nb2))) continue;
            perm[pos] = w;
            rec(pos + 1, used | (1 << w), b, nb2);
        }
    }
};
}  // namespace

Code canonical(const Pat &p, int *perm) {
    CanonSearch s;
    s.p = &p;
    s.n = p.n;
    for (int i = 0; i < p.n; i++) s.slab[i] = p.lab[i];
    std::sort(s.slab, s.slab + p.n);
    s.have = false;
    s.best_bits = 0;
    s.total_bits = p.n * (p.n - 1) / 2;
    for (int w = 0; w < p.n; w++) {
        s.twin_below[w] = 0;
        for (int u = 0; u < w; u++)
            if (p.lab[u] == p.lab[w] &&
                (p.adj[u] & ~(uint8_t)(1u << w)) == (p.adj[w] & ~(uint8_t)(1u << u)))
                s.twin_below[w] |= 1u << u;
    }
    s.rec(0, 0, 0, 0);
    Code c;
    c.n = p.n;
    for (int i = 0; i < p.n; i++) c.lab[i] = s.slab[i];
    c.bits = s.best_bits;
    if (perm) memcpy(perm, s.best_perm, sizeof(int) * p.n);
    return c;
}

// Directed patterns: the code of an order is (labels in order, then for columns j = 1..n-1 and rows
// i = 0..j-1 two bits: "no arc i -> j", "no arc j -> i"), the canonical order the one with the
// lexicographically smallest code; positions are filled left to right with the label of each
// position forced (sorted label multiset) and prefixes that exceed the best code's are pruned.
namespace {
struct DCanonSearch {
    const Pat *p;
    int n;
    int32_t slab[MAXN];
    int perm[MAXN];
    int best_perm[MAXN];
    uint64_t best_bits;
    bool have;
    int total_bits;

    void rec(int pos, int used, uint64_t bits, int nb) {
        if (pos == n) {
            if (!have || bits < best_bits) {
                best_bits = bits;
                memcpy(best_perm, perm, sizeof(int) * n);
                have = true;
            }
            return;
        }
        for (int w = 0; w < n; w++) {
            if ((used >> w & 1) || p->lab[w] != slab[pos]) continue;
            uint64_t b = bits;
            for (int i = 0; i < pos; i++) {
                b = (b << 1) | (((p->out[perm[i]] >> w) & 1) ? 0u : 1u);
                b = (b << 1) | (((p->out[w] >> perm[i]) & 1) ? 0u : 1u);
            }
            const int nb2 = nb + 2 * pos;
            if (have && nb2 > 0 && b > (best_bits >> (total_bits - nb2))) continue;
            perm[pos] = w;
            rec(pos + 1, used | (1 << w), b, nb2);
        }
    }
};
}  // namespace

void canonical_directed(const Pat &p, int *perm, uint64_t *bits) {
    DCanonSearch s;
    s.p = &p;
    s.n = p.n;
    for (int i = 0; i < p.n; i++) s.slab[i] = p.lab[i];
    std::sort(s.slab, s.slab + p.n);
    s.have = false;
    s.best_bits = 0;
    s.total_bits = p.n * (p.n - 1);
    s.rec(0, 0, 0, 0);
    memcpy(perm, s.best_perm, sizeof(int) * p.n);
    if (bits) *bits = s.best_bits;
}

Pat pat_of_code(const Code &c) {
    Pat p;
    p.n = c.n;
    for (int i = 0; i < c.n; i++) p.lab[i] = c.lab[i];
    int t = c.n * (c.n - 1) / 2 - 1;
    for (int j = 1; j < c.n; j++)
        for (int i = 0; i < j; i++, t--)
            if (!((c.bits >> t) & 1)) {
                p.adj[i] |= (uint8_t)(1 << j);
                p.adj[j] |= (uint8_t)(1 << i);
            }
    return p;
}

// ---------------------------------------------------------------- automorphisms and orbits
namespace {
struct AutSearch {
    const Pat *p;
    std::vector<std::array<int8_t, MAXN>> *out;
    size_t limit;
    int img[MAXN];
    void rec(int pos, int used) {
        if (out->size() >= limit) return;
        if (pos == p->n) {
            std::array<int8_t, MAXN> a{};
            for (int i = 0; i < p->n; i++) a[i] = (int8_t)img[i];
            out->push_back(a);
            return;
        }
        for (int w = 0; w < p->n; w++) {
            if (used >> w & 1) continue;
            if (p->lab[w] != p->lab[pos]) continue;
            if (__builtin_popcount(p->adj[w]) != __builtin_popcount(p->adj[pos])) continue;
            bool ok = true;
            for (int i = 0; i < pos && ok; i++)
                if (has(*p, i, pos) != has(*p, img[i], w)) ok = false;
            if (p->directed)  // arcs keep their direction
                for (int i = 0; i < pos && ok; i++)
                    if (((p->out[i] >> pos) & 1) != ((p->out[img[i]] >> w) & 1) ||
                        ((p->out[pos] >> i) & 1) != ((p->out[w] >> img[i]) & 1))
                        ok = false;
            if (!ok) continue;
            img[pos] = w;
            rec(pos + 1, used | (1 << w));
        }
    }
};
}  // namespace

void automorphisms(const Pat &p, std::vector<std::array<int8_t, MAXN>> *out, size_t limit) {
    AutSearch s;
    s.p = &p;
    s.out = out;
    s.limit = limit;
    s.rec(0, 0);
}

void orbits(const Pat &p, int *orb) {
    // u ~ v iff some automorphism maps u to v; orb[v] = smallest vertex of v's orbit
    std::vector<std::array<int8_t, MAXN>> all;
    automorphisms(p, &all, SIZE_MAX);
    for (int v = 0; v < p.n; v++) {
        orb[v] = v;
        for (auto &a : all) orb[v] = std::min(orb[v], (int)a[v]);
    }
}

// Level masks of a matching order over canonical pattern q.
static LevelPlan plan_of_order(const Pat &q, const int *order) {
    LevelPlan L;
    memset(&L, 0, sizeof L);
    for (int i = 0; i < q.n; i++) {
        L.vert[i] = (uint8_t)order[i];
        L.lab[i] = (uint8_t)q.lab[order[i]];
        uint8_t bm = 0, im = 0;
        uint16_t bd = 0;
        for (int j = 0; j < i; j++) {
            if (has(q, order[j], order[i])) {
                bm |= (uint8_t)(1 << j);
                if (q.directed) {
                    const bool fwd = (q.out[order[j]] >> order[i]) & 1, back = (q.out[order[i]] >> order[j]) & 1;
                    const int d = fwd && back ? DIR_MUT : fwd ? DIR_OUT : DIR_IN;
                    bd |= (uint16_t)(d << (2 * j));
                }
            }
            if (q.lab[order[j]] == q.lab[order[i]]) im |= (uint8_t)(1 << j);
        }
        L.bdir[i] = bd;
        L.bmask[i] = bm;
        L.injmask[i] = im;
        L.deg[i] = (uint8_t)__builtin_popcount(q.adj[order[i]]);
    }
    return L;
}

LevelPlan level_plan(const Pat &q, int first) {
    int order[MAXN];
    int visited = 1 << first;
    order[0] = first;
    for (int k = 1; k < q.n; k++) {
        int reach = 0;
        for (int u = 0; u < q.n; u++)
            if (visited >> u & 1) reach |= q.adj[u];
        reach &= ~visited;
        const int pick = __builtin_ctz((unsigned)reach);  // smallest unvisited position adjacent to visited
        order[k] = pick;
        visited |= 1 << pick;
    }
    return plan_of_order(q, order);
}


// ---------------------------------------------------------------- tau and plans
int64_t tau_exact(int64_t sigma, int64_t lam_num, int64_t lam_den, int n) {
    __int128 top = (__int128)sigma * ((__int128)(n - 1) * lam_num + lam_den);
    __int128 bot = (__int128)n * lam_den;
    return (int64_t)(top / bot);
}

// The or-ed mode flags: the remaining base mode must be FLEXIS_MODE_EARLY or FLEXIS_MODE_FULL.
static bool parse_mode(int mode, Plan &P) {
    P.want_mni = (mode & FLEXIS_MODE_NO_MNI) ? 0 : 1;
    P.count_maps = (mode & FLEXIS_MODE_COUNT_MAPS) ? 1 : 0;
    P.skip_mis = (mode & FLEXIS_MODE_NO_MIS) ? 1 : 0;
    P.exact_mis = (mode & FLEXIS_MODE_EXACT_MIS) ? 1 : 0;
    mode &= ~(FLEXIS_MODE_NO_MNI | FLEXIS_MODE_COUNT_MAPS | FLEXIS_MODE_NO_MIS | FLEXIS_MODE_EXACT_MIS);
    P.mode = mode;
    if (!P.want_mni) P.flags |= FLEXIS_FLAG_MNI_SKIPPED;
    if (P.skip_mis) P.flags |= FLEXIS_FLAG_MIS_SKIPPED;
    return mode == FLEXIS_MODE_EARLY || mode == FLEXIS_MODE_FULL;
}

int compile_plan(const HostGraph &g, const flexis_pattern &pat, int64_t sigma, int64_t lam_num,
                 int64_t lam_den, int mode, Plan &P) {
    memset(&P, 0, sizeof P);
    P.status = FLEXIS_E_INVALID;
    P.n = pat.n;
    P.sigma = sigma;
    const bool mode_ok = parse_mode(mode, P);
    mode = P.mode;
    if (pat.n < 2 || pat.n > MAXN || pat.m < 0 || pat.labels == nullptr ||
        (pat.m > 0 && pat.edges == nullptr))
        return FLEXIS_E_INVALID;
    if (sigma < 1 || lam_den <= 0 || lam_num < 0 || lam_num > lam_den) return FLEXIS_E_INVALID;
    if (!mode_ok) return FLEXIS_E_INVALID;
    Pat p;
    p.n = pat.n;
    for (int i = 0; i < pat.n; i++) {
        if (pat.labels[i] < 0) return FLEXIS_E_INVALID;
        p.lab[i] = pat.labels[i];
    }
    p.directed = g.directed != 0;  // on a directed graph an edge (a, b) is the arc a -> b
    for (int e = 0; e < pat.m; e++) {
        int a = pat.edges[2 * e], b = pat.edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= pat.n || b >= pat.n || a == b) return FLEXIS_E_INVALID;
        p.adj[a] |= (uint8_t)(1 << b);
        p.adj[b] |= (uint8_t)(1 << a);
        p.out[a] |= (uint8_t)(1 << b);
    }
    if (!connected(p)) return FLEXIS_E_INVALID;
    P.n_edges = edge_count(p);
    P.tau = tau_exact(sigma, lam_num, lam_den, pat.n);
    int64_t c = P.tau > 1 ? P.tau : 1;
    P.cap = mode == FLEXIS_MODE_EARLY ? c : CAP_INF;
    P.status = FLEXIS_OK;
    // labels -> ranks; an absent label means no map at all
    for (int i = 0; i < pat.n; i++) {
        int32_t r = pat.labels[i] < g.nl_ids ? g.rank_of[pat.labels[i]] : -1;
        if (r < 0) {
            P.flags |= FLEXIS_FLAG_ABSENT_LABEL;
            P.root_begin = P.root_end = 0;
            P.n_orb = 0;
            return FLEXIS_OK;
        }
        p.lab[i] = r;
    }
    if (!p.directed) {
        fill_plan(g, canonical(p, nullptr), P);
        return FLEXIS_OK;
    }
    int perm[MAXN];
    canonical_directed(p, perm, nullptr);
    Pat q;
    q.n = p.n;
    q.directed = true;
    for (int i = 0; i < p.n; i++) {
        q.lab[i] = p.lab[perm[i]];
        for (int j = 0; j < p.n; j++) {
            if ((p.adj[perm[i]] >> perm[j]) & 1) q.adj[i] |= (uint8_t)(1 << j);
            if ((p.out[perm[i]] >> perm[j]) & 1) q.out[i] |= (uint8_t)(1 << j);
        }
    }
    P.code_n = q.n;
    for (int i = 0; i < q.n; i++) P.code_lab[i] = (uint8_t)q.lab[i];
    P.code_bits = 0;  // directed codes are not reported
    fill_plan_pat(g, q, P);
    return FLEXIS_OK;
}

// Matching orders, label slices and (when MNI is wanted) orbit plans of a canonical pattern
// whose labels are ranks of g.
void fill_plan(const HostGraph &g, const Code &code, Plan &P) {
    P.code_n = code.n;
    for (int i = 0; i < code.n; i++) P.code_lab[i] = (uint8_t)code.lab[i];
    P.code_bits = code.bits;
    fill_plan_pat(g, pat_of_code(code), P);
}

void fill_plan_pat(const HostGraph &g, const Pat &q, Plan &P) {
    for (int u = 0; u < q.n; u++) {
        P.cadj[u] = q.adj[u];
        for (int w = 0; w < q.n; w++)
            if ((q.adj[u] >> w & 1) && q.lab[w] < 64) P.need[u] |= 1ull << q.lab[w];
        P.lab_begin[u] = g.lab_ptr[q.lab[u]];
        P.lab_end[u] = g.lab_ptr[q.lab[u] + 1];
    }
    P.greedy = level_plan(q, 0);
    P.root_begin = P.lab_begin[0];
    P.root_end = P.lab_end[0];
    P.n_orb = 0;
    if (!P.want_mni) return;
    int orb[MAXN];
    orbits(q, orb);
    int k = 0;
    for (int u = 0; u < q.n; u++) {
        if (orb[u] != u) continue;
        P.orb[k] = level_plan(q, u);  // orb[k].vert[0] == u
        k++;
    }
    P.n_orb = k;
}

// Plan of a pattern already in canonical form over the graph's label ranks (mining candidates).
int compile_code(const HostGraph &g, const Code &code, int64_t sigma, int64_t lam_num,
                 int64_t lam_den, int mode, Plan &P) {
    memset(&P, 0, sizeof P);
    P.n = code.n;
    P.sigma = sigma;
    if (!parse_mode(mode, P)) {
        P.status = FLEXIS_E_INVALID;
        return FLEXIS_E_INVALID;
    }
    mode = P.mode;
    P.n_edges = edge_count(pat_of_code(code));
    P.tau = tau_exact(sigma, lam_num, lam_den, code.n);
    const int64_t c = P.tau > 1 ? P.tau : 1;
    P.cap = mode == FLEXIS_MODE_EARLY ? c : CAP_INF;
    P.status = FLEXIS_OK;
    fill_plan(g, code, P);
    return FLEXIS_OK;
}

// ---------------------------------------------------------------- candidate generation
// Algorithm 2: core groups (Sec. 2.3.3) -> merge every pair of core graphs of a group under
// every automorphism of the common core Gamma (Algorithm 3 returns either all automorphisms
// or the identity; using all of them always is a superset that duplicate removal reduces to
// the same set) -> cliques by a third core graph plus the post-check that every (k-1)-sub-clique
// is frequent (Algorithm 4) -> RemoveDuplicates by canonical code.
namespace {
struct CoreEntry {
    int32_t lab;    // marked vertex label
    uint8_t mask;   // marked vertex attachment over the core's canonical positions
    bool operator<(const CoreEntry &o) const { return lab != o.lab ? lab < o.lab : mask < o.mask; }
    bool operator==(const CoreEntry &o) const { return lab == o.lab && mask == o.mask; }
};

struct Group {
    Code core;
    std::vector<std::array<int8_t, MAXN>> aut;
    std::vector<CoreEntry> entries;
};

uint8_t map_mask(uint8_t m, const std::array<int8_t, MAXN> &a, int n) {
    uint8_t r = 0;
    for (int i = 0; i < n; i++)
        if (m >> i & 1) r |= (uint8_t)(1 << a[i]);
    return r;
}
}  // namespace

void generate_candidates(const std::vector<Code> &F, int max_edges, std::vector<Code> &out,
                         int threads) {
    out.clear();
    if (F.empty()) return;
    std::unordered_set<Code, CodeHash> Fset(F.begin(), F.end());
    const int T = std::max(1, threads);
    auto parallel = [&](size_t count, const std::function<void(int, size_t, size_t)> &body) {
        std::vector<std::thread> th;
        const size_t per = (count + (size_t)T - 1) / (size_t)T;
        for (int t = 1; t < T; t++) {
            const size_t lo = std::min(count, per * (size_t)t), hi = std::min(count, lo + per);
            th.emplace_back(body, t, lo, hi);
        }
        body(0, 0, std::min(count, per));
        for (auto &x : th) x.join();
    };
    // core groups: every (member, removed vertex) gives a core in canonical form and the removed
    // vertex's label and attachment over the core's canonical positions; computed per thread,
    // then grouped by sorting on the core
    struct CoreRec {
        Code core;
        CoreEntry e;
    };
    std::vector<size_t> first((size_t)F.size() + 1, 0);
    for (size_t f = 0; f < F.size(); f++) first[f + 1] = first[f] + (size_t)F[f].n;
    std::vector<CoreRec> recs(first.back());
    parallel(F.size(), [&](int, size_t lo, size_t hi) {
        for (size_t f = lo; f < hi; f++) {
            const Pat P = pat_of_code(F[f]);
            for (int x = 0; x < P.n; x++) {
                Pat core;
                core.n = P.n - 1;
                int pos[MAXN], k = 0;
                for (int i = 0; i < P.n; i++)
                    if (i != x) pos[k++] = i;
                for (int i = 0; i < core.n; i++) {
                    core.lab[i] = P.lab[pos[i]];
                    for (int j = 0; j < core.n; j++)
                        if (has(P, pos[i], pos[j])) core.adj[i] |= (uint8_t)(1 << j);
                }
                int perm[MAXN];
                const Code cc = canonical(core, perm);
                uint8_t mask = 0;
                for (int cp = 0; cp < core.n; cp++)
                    if (has(P, x, pos[perm[cp]])) mask |= (uint8_t)(1 << cp);
                recs[first[f] + (size_t)x] = CoreRec{cc, CoreEntry{P.lab[x], mask}};
            }
        }
    });
    // group: records are spread over buckets by the core's hash (equal cores share a bucket),
    // each bucket is sorted and cut into groups in parallel; the order of the groups does not
    // matter (every group's candidates end in the sorted, deduplicated output)
    const size_t nb = (size_t)T * 8;
    std::vector<size_t> bstart(nb + 1, 0);
    std::vector<uint32_t> bucket_of(recs.size());
    CodeHash hasher;
    for (size_t i = 0; i < recs.size(); i++) {
        bucket_of[i] = (uint32_t)(hasher(recs[i].core) % nb);
        bstart[bucket_of[i] + 1]++;
    }
    for (size_t b = 0; b < nb; b++) bstart[b + 1] += bstart[b];
    std::vector<CoreRec> byb(recs.size());
    {
        std::vector<size_t> fill(bstart.begin(), bstart.end() - 1);
        for (size_t i = 0; i < recs.size(); i++) byb[fill[bucket_of[i]]++] = recs[i];
    }
    std::vector<CoreRec>().swap(recs);
    std::vector<std::vector<Group>> bgroups(nb);
    {
        std::atomic<size_t> next_b{0};
        auto worker = [&] {
            for (size_t b; (b = next_b.fetch_add(1)) < nb;) {
                auto lo = byb.begin() + (ptrdiff_t)bstart[b], hi = byb.begin() + (ptrdiff_t)bstart[b + 1];
                std::sort(lo, hi, [](const CoreRec &x, const CoreRec &y) {
                    if (!(x.core == y.core)) return x.core < y.core;
                    return x.e < y.e;
                });
                for (auto it = lo; it != hi; ++it) {
                    if (it == lo || !(it->core == (it - 1)->core)) bgroups[b].push_back(Group{it->core, {}, {}});
                    bgroups[b].back().entries.push_back(it->e);
                }
            }
        };
        std::vector<std::thread> th;
        for (int t = 1; t < T; t++) th.emplace_back(worker);
        worker();
        for (auto &x : th) x.join();
    }
    std::vector<CoreRec>().swap(byb);
    std::vector<Group> groups;
    for (auto &v : bgroups)
        for (auto &gr : v) groups.push_back(std::move(gr));
    std::vector<int32_t> labels;
    for (const Code &c : F)
        for (int i = 0; i < c.n; i++) labels.push_back(c.lab[i]);
    std::sort(labels.begin(), labels.end());
    labels.erase(std::unique(labels.begin(), labels.end()), labels.end());

    std::vector<std::vector<Code>> part((size_t)std::max(1, threads));
    std::atomic<size_t> next{0};
    auto work = [&](int tid) {
        std::vector<Code> &local = part[(size_t)tid];
        size_t limit = (size_t)1 << 22;
        for (;;) {
            size_t gi = next.fetch_add(1);
            if (gi >= groups.size()) break;
            Group &G = groups[gi];
            Pat core = pat_of_code(G.core);
            std::vector<std::array<int8_t, MAXN>> aut;
            automorphisms(core, &aut, SIZE_MAX);
            // entries up to Aut(core): keep one representative (minimum mask image)
            std::vector<CoreEntry> ent;
            for (auto e : G.entries) {
                uint8_t best = e.mask;
                for (auto &a : aut) best = std::min(best, map_mask(e.mask, a, core.n));
                ent.push_back(CoreEntry{e.lab, best});
            }
            std::sort(ent.begin(), ent.end());
            ent.erase(std::unique(ent.begin(), ent.end()), ent.end());
            int kc = core.n;
            int core_edges = edge_count(core);
            for (size_t a = 0; a < ent.size(); a++)
                for (size_t b = a; b < ent.size(); b++)
                    for (auto &al : aut) {
                        uint8_t mb = map_mask(ent[b].mask, al, kc);
                        int m = core_edges + __builtin_popcount(ent[a].mask) + __builtin_popcount(mb);
                        if (max_edges > 0 && m > max_edges) continue;
                        Pat P = core;
                        P.n = kc + 2;
                        int x = kc, y = kc + 1;
                        P.lab[x] = ent[a].lab;
                        P.lab[y] = ent[b].lab;
                        P.adj[x] = ent[a].mask;
                        P.adj[y] = mb;
                        for (int i = 0; i < kc; i++) {
                            if (ent[a].mask >> i & 1) P.adj[i] |= (uint8_t)(1 << x);
                            if (mb >> i & 1) P.adj[i] |= (uint8_t)(1 << y);
                        }
                        if (!connected(P)) continue;
                        local.push_back(canonical(P, nullptr));
                    }
            if (local.size() > limit) {  // bound the repeats held
                std::sort(local.begin(), local.end());
                local.erase(std::unique(local.begin(), local.end()), local.end());
                limit = std::max(limit, 2 * local.size());
            }
        }
        std::sort(local.begin(), local.end());
        local.erase(std::unique(local.begin(), local.end()), local.end());
    };
    {
        std::vector<std::thread> th;
        for (int t = 1; t < T; t++) th.emplace_back(work, t);
        work(0);
        for (auto &t : th) t.join();
    }
    std::vector<Code> cliques;
    // cliques (Algorithm 4 + post-check): a k-clique whose every (k-1)-sub-clique is frequent
    for (const Code &c : F) {
        Pat Q = pat_of_code(c);
        int kq = Q.n;
        if (edge_count(Q) != kq * (kq - 1) / 2) continue;
        if (kq + 1 > MAXN) continue;
        int m = kq * (kq + 1) / 2;
        if (max_edges > 0 && m > max_edges) continue;
        for (int32_t l : labels) {
            Pat P = Q;
            P.n = kq + 1;
            P.lab[kq] = l;
            P.adj[kq] = (uint8_t)((1 << kq) - 1);
            for (int i = 0; i < kq; i++) P.adj[i] |= (uint8_t)(1 << kq);
            bool ok = true;
            for (int u = 0; u < P.n && ok; u++) {
                Pat R;
                R.n = P.n - 1;
                int k = 0;
                for (int i = 0; i < P.n; i++) {
                    if (i == u) continue;
                    R.lab[k] = P.lab[i];
                    k++;
                }
                for (int i = 0; i < R.n; i++) R.adj[i] = (uint8_t)(((1 << R.n) - 1) & ~(1 << i));
                if (!Fset.count(canonical(R, nullptr))) ok = false;
            }
            if (ok) cliques.push_back(canonical(P, nullptr));
        }
    }
    std::sort(cliques.begin(), cliques.end());
    part.push_back(std::move(cliques));
    // union of the sorted runs (one per thread, plus the cliques): the key space is cut at
    // splitters taken from the largest run; each piece is a k-way merge that drops repeats, run
    // in parallel, and the pieces are concatenated in key order (sorted and unique overall)
    size_t big = 0;
    for (size_t r = 0; r < part.size(); r++)
        if (part[r].size() > part[big].size()) big = r;
    std::vector<Code> split;  // piece p holds keys in [split[p-1], split[p])
    const size_t pieces = part[big].size() > 4096 ? (size_t)T * 4 : 1;
    for (size_t p = 1; p < pieces; p++) split.push_back(part[big][part[big].size() * p / pieces]);
    split.erase(std::unique(split.begin(), split.end()), split.end());
    const size_t np = split.size() + 1;
    std::vector<std::vector<Code>> merged(np);
    auto merge_piece = [&](size_t p) {
        std::vector<std::pair<size_t, size_t>> rng(part.size());  // [begin, end) of each run
        for (size_t r = 0; r < part.size(); r++) {
            const auto &v = part[r];
            const size_t b = p == 0 ? 0 : (size_t)(std::lower_bound(v.begin(), v.end(), split[p - 1]) - v.begin());
            const size_t e = p + 1 == np ? v.size() : (size_t)(std::lower_bound(v.begin(), v.end(), split[p]) - v.begin());
            rng[r] = {b, e};
        }
        auto run_less = [&](size_t a, size_t b) { return part[b][rng[b].first] < part[a][rng[a].first]; };
        std::vector<size_t> heap;
        size_t total = 0;
        for (size_t r = 0; r < part.size(); r++)
            if (rng[r].first < rng[r].second) {
                heap.push_back(r);
                total += rng[r].second - rng[r].first;
            }
        std::vector<Code> &o = merged[p];
        o.reserve(total);
        std::make_heap(heap.begin(), heap.end(), run_less);
        while (!heap.empty()) {
            std::pop_heap(heap.begin(), heap.end(), run_less);
            const size_t r = heap.back();
            const Code &c = part[r][rng[r].first];
            if (o.empty() || !(o.back() == c)) o.push_back(c);
            if (++rng[r].first < rng[r].second) std::push_heap(heap.begin(), heap.end(), run_less);
            else heap.pop_back();
        }
    };
    {
        std::atomic<size_t> next_piece{0};
        auto worker = [&] {
            for (size_t p; (p = next_piece.fetch_add(1)) < np;) merge_piece(p);
        };
        std::vector<std::thread> th;
        for (int t = 1; t < T; t++) th.emplace_back(worker);
        worker();
        for (auto &x : th) x.join();
    }
    size_t total = 0;
    for (auto &v : merged) total += v.size();
    out.reserve(total);
    for (auto &v : merged) out.insert(out.end(), v.begin(), v.end());
}

}  // namespace fx
