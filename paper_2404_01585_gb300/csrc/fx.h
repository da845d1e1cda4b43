// Internal types of the FLEXIS GB300 library (host runtime + kernels).
#pragma once
#include <cstddef>
#include <cstdint>
#include <array>
#include <string>
#include <vector>

#include "../../include/flexis.h"

namespace fx {

constexpr int MAXN = 8;                 // largest pattern (vertices)
constexpr int64_t CAP_INF = INT64_MAX;  // "no cap" (FULL mode)
constexpr uint64_t DEFAULT_SEED = 0x5EEDull;
constexpr uint32_t RUN_SENTINEL_LABEL = 0xFFu;

// A matching order over the canonical pattern (Sec. 3.2.2 matcher, depth-first by level).
// Level i binds canonical vertex vert[i]; its candidates must carry rank label lab[i], be
// adjacent to the data vertices bound at every level j with bit j of bmask[i], and differ from
// those bound at the levels in injmask[i] (earlier levels with the same label).
struct LevelPlan {
    uint8_t lab[MAXN];
    uint8_t bmask[MAXN];
    uint8_t injmask[MAXN];
    uint8_t vert[MAXN];
    uint8_t deg[MAXN];     // pattern degree of the vertex bound at level i
    uint16_t bdir[MAXN];   // directed patterns: 2 bits per backward level j (bits 2j..2j+1): the
                           // list of the vertex bound at j that holds level i's candidates --
                           // DIR_OUT (arc j -> i), DIR_IN (arc i -> j) or DIR_MUT (both arcs)
};
enum : int { DIR_OUT = 0, DIR_IN = 1, DIR_MUT = 2 };

// Compiled pattern (host pattern compiler output; plain bytes, device readable).
struct Plan {
    int32_t n;
    int32_t status;      // FLEXIS_OK or an error for this pattern
    uint32_t flags;      // FLEXIS_FLAG_*
    int32_t n_orb;       // automorphism orbits (MNI representatives)
    int64_t sigma, tau, cap;  // cap: EARLY max(tau,1); FULL CAP_INF
    int32_t mode;
    int32_t root_begin, root_end;  // greedy roots: slice of the label index
    int32_t n_edges;
    LevelPlan greedy;               // matching order rooted at canonical vertex 0
    LevelPlan orb[MAXN];            // matching order rooted at each orbit representative
    uint8_t code_lab[MAXN];         // canonical code: rank labels in canonical order
    uint8_t cadj[MAXN];             // canonical pattern adjacency rows (bit j: i ~ j)
    uint32_t code_bits;             // canonical code: adjacency bits
    int32_t code_n;
    int32_t want_mni;               // 0 under FLEXIS_MODE_NO_MNI
    int32_t lab_begin[MAXN], lab_end[MAXN];  // label-index slice of each canonical vertex's label
    uint64_t need[MAXN];            // rank labels (< 64) of each canonical vertex's neighbours
    int32_t count_maps;             // FLEXIS_MODE_COUNT_MAPS: enumerate and count all maps
    int32_t skip_mis;               // FLEXIS_MODE_NO_MIS: no greedy phase
    int32_t exact_mis;              // FLEXIS_MODE_EXACT_MIS: maximum independent set of the instances
    int32_t decide_only;            // mining: an infrequent pattern may stop as soon as it cannot
                                    // reach c (its mis is then a lower bound; only frequent
                                    // patterns are kept)
};
static_assert(sizeof(Plan) <= sizeof(flexis_plan), "plan must fit flexis_plan");

// Per-vertex record, one 32-byte sector: adjacency offset, label-run offset, degree,
// (number of label runs << 8 | rank label), and the set of rank labels < 64 found among the
// neighbours (a one-hop filter: a pattern vertex whose neighbours need label l cannot be hosted
// by a data vertex without a neighbour of label l).
struct alignas(32) VRec {
    uint32_t adj;
    uint32_t run;
    uint32_t deg;
    uint32_t meta;
    uint64_t nbr_labels;
    uint64_t pad;
};

// Host copy of the data graph layout (built on the host, mirrored on the device).
struct HostGraph {
    int64_t nv = 0;
    int32_t directed = 0;               // vrec holds 3 * nv records: out, in and mutual lists
    int32_t nl_ids = 0;                 // label ids 0..nl_ids-1
    int32_t nl = 0;                     // labels present (ranks 0..nl-1)
    std::vector<int32_t> rank_of;       // [nl_ids] rank or -1
    std::vector<int32_t> label_of_rank; // [nl]
    std::vector<VRec> vrec;             // [nv]
    std::vector<uint32_t> runs;         // per vertex: runs (lab<<24 | rel start) + sentinel
    std::vector<int32_t> adj;           // sorted by (rank label, id) per vertex
    std::vector<int32_t> lab_vtx;       // vertices by (rank, H(seed,v), v)
    std::vector<int32_t> lab_ptr;       // [nl+1]
    std::vector<std::pair<int32_t, int32_t>> label_pairs;  // rank pairs (a<=b) on data edges
    int64_t n_arcs = 0;
    int64_t self_loops = 0, duplicates = 0;
    int32_t max_degree = 0;
    uint64_t seed = DEFAULT_SEED;
};

uint64_t root_hash(uint64_t seed, int64_t r);

// host graph construction (graph.cpp)
// Label tables of a graph (nl_ids, nl, rank_of, label_of_rank, lab_ptr) and the rank of every
// vertex (rk[max(nv, 1)]); FLEXIS_E_INVALID for a negative label, FLEXIS_E_UNSUPPORTED for 255
// or more labels present.
int label_ranks(int64_t nv, const int32_t *labels, HostGraph &g, std::vector<uint8_t> &rk);
int build_host_graph(int64_t nv, const int32_t *labels, int64_t ne, const int32_t *src,
                     const int32_t *dst, uint64_t seed, int id_order, HostGraph &out,
                     int directed = 0);

// ------------------------------------------------------------------ patterns (pattern.cpp)
struct Pat {  // small labelled graph, adjacency as bit rows
    int n = 0;
    int32_t lab[MAXN] = {0};
    uint8_t adj[MAXN] = {0};  // bit j of adj[i]: i ~ j (for a directed pattern: an arc either way)
    uint8_t out[MAXN] = {0};  // directed pattern: bit j of out[i]: arc i -> j
    bool directed = false;
};

struct Code {  // canonical code: (n, labels, bits)
    int n = 0;
    int32_t lab[MAXN] = {0};
    uint32_t bits = 0;
    bool operator<(const Code &o) const;
    bool operator==(const Code &o) const;
};

struct CodeHash {
    size_t operator()(const Code &c) const;
};

// canonical form: returns the code; perm[p] = vertex of `p` at canonical position p
Code canonical(const Pat &p, int *perm);
// canonical vertex order of a directed pattern (see pattern.cpp); *bits gets its 2-bit-per-pair
// code
void canonical_directed(const Pat &p, int *perm, uint64_t *bits);
Pat pat_of_code(const Code &c);
bool connected(const Pat &p);
int edge_count(const Pat &p);
// all automorphisms of p (as permutations), capped at `limit`
void automorphisms(const Pat &p, std::vector<std::array<int8_t, MAXN>> *out, size_t limit);
// orbit id per vertex (smallest vertex of its orbit)
void orbits(const Pat &p, int *orb);
// matching order rooted at `first` over canonical pattern q
LevelPlan level_plan(const Pat &q, int first);

// pattern compile: labels as graph label ids
void fill_plan(const HostGraph &g, const Code &code, Plan &P);
void fill_plan_pat(const HostGraph &g, const Pat &canonical_pattern, Plan &P);
int compile_code(const HostGraph &g, const Code &code, int64_t sigma, int64_t lam_num,
                 int64_t lam_den, int mode, Plan &P);
int compile_plan(const HostGraph &g, const flexis_pattern &pat, int64_t sigma, int64_t lam_num,
                 int64_t lam_den, int mode, Plan &out);
int64_t tau_exact(int64_t sigma, int64_t lam_num, int64_t lam_den, int n);

// candidate generation (Algorithms 2-4): F given as canonical codes (labels as given)
void generate_candidates(const std::vector<Code> &F, int max_edges, std::vector<Code> &out,
                         int threads);

}  // namespace fx
