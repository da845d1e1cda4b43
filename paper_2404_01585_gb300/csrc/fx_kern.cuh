// Device-side pieces shared by the kernels of the support-evaluation path (kernels.cu) and of
// the map enumerator, overlap graph and exact MIS (enumerate.cu): the resident graph view, the
// warp depth-first search over label slices, block scans, and the device graph with its
// evaluation workspace.
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <vector>

#include "fx_dev.h"

namespace fx {

#define FULLMASK 0xFFFFFFFFu

struct DevGraphView {
    const VRec *vrec;
    const uint32_t *runs;
    const int32_t *adj;
    const int32_t *lab_vtx;
    int64_t nv;
    int32_t words;  // used-bitmap words per pattern
    int64_t dstride;  // directed graphs: nv (records of the out, in and mutual lists follow each
                      // other); undirected: 0 (every direction reads the one neighbour list)
};

// ------------------------------------------------------------------ warp depth-first search
struct WarpState {
    int32_t t[MAXN];                    // data vertex bound at each level
    uint32_t lo[MAXN], hi[MAXN];        // driver slice of each level
    uint32_t pos[MAXN], base[MAXN], mask[MAXN];
    uint32_t conf[MAXN];                // backjump conflict set of each level (bits of levels)
    uint32_t clo[MAXN][MAXN - 1], chi[MAXN][MAXN - 1];  // further slices (membership tests)
    int32_t nchk[MAXN];
    int32_t level;                      // level at suspension
    int32_t floor;                      // lowest level this search may rebind (1: whole root)
    // --- the fields above are the resumable search state (DFS_SAVE_WORDS words)
    unsigned long long need[MAXN];      // neighbour labels each canonical vertex needs
    LevelPlan L;
    int32_t n;
    int32_t pad[1];
    // slice cache: the slice of level i's candidates in the list of the vertex bound at level b
    // depends on that vertex only (label and list are fixed by the plan), so it is looked up
    // once per vertex bound there; sc_v[i][b] is the vertex it was looked up for (-1: none)
    int32_t sc_v[MAXN][MAXN];
    uint32_t sc_lo[MAXN][MAXN], sc_hi[MAXN][MAXN];
    // per-warp totals of the algorithmic work (kept by lane 0, out of the registers)
    unsigned long long acc_scanned, acc_bound, acc_maps;
};

__device__ __forceinline__ bool used_bit(const uint32_t *used, int32_t v) {
    return (__ldcg(used + (v >> 5)) >> (v & 31)) & 1u;
}

// Slice of v's neighbours in list `dir` (DIR_OUT / DIR_IN / DIR_MUT) carrying rank label `lab`
// (warp-cooperative: one load of up to 32 label runs, ballot on the label).  Returns an empty
// slice when the label is absent.
__device__ __forceinline__ void find_slice(const DevGraphView &G, int32_t v, uint32_t lab, uint32_t dir,
                                           uint32_t &lo, uint32_t &hi, unsigned long long &bytes) {
    const int lane = threadIdx.x & 31;
    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(G.vrec + (int64_t)dir * G.dstride + v));
    bytes += 16;
    const uint32_t adj = r.x, run = r.y, nrun = r.w >> 8;
    lo = hi = 0;
    for (uint32_t j0 = 0; j0 < nrun; j0 += 32) {
        const uint32_t j = j0 + lane;
        const uint32_t e = (j <= nrun) ? __ldg(G.runs + run + j) : 0xFFFFFFFFu;
        const uint32_t nx = __shfl_down_sync(FULLMASK, e, 1);
        bytes += 4ull * min(32u, nrun + 1 - j0);
        const bool hit = (j < nrun) && ((e >> 24) == lab);
        const unsigned b = __ballot_sync(FULLMASK, hit);
        if (b) {
            const int s = __ffs(b) - 1;
            const uint32_t es = __shfl_sync(FULLMASK, e, s);
            uint32_t en = __shfl_sync(FULLMASK, nx, s);
            if (s == 31) en = __ldg(G.runs + run + j0 + 32);
            lo = adj + (es & 0xFFFFFFu);
            hi = adj + (en & 0xFFFFFFu);
            return;
        }
        const uint32_t last = __shfl_sync(FULLMASK, e, 31);
        if ((last >> 24) > lab) return;  // runs are sorted by label
    }
}

__device__ __forceinline__ bool contains(const int32_t *adj, uint32_t lo, uint32_t hi, int32_t c,
                                         uint32_t &probes) {
    uint32_t a = lo, b = hi;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        probes++;
        if (__ldg(adj + m) < c) a = m + 1; else b = m;
    }
    if (a >= hi) return false;
    probes++;
    return __ldg(adj + a) == c;
}

// Prepare level i: slices of the bound neighbours at every backward level; the shortest one
// drives the scan, the others are membership tests.  False if some slice is empty.
__device__ __forceinline__ bool enter_level(const DevGraphView &G, WarpState &W, int i,
                                            unsigned long long &bytes) {
    const int lane = threadIdx.x & 31;
    const uint32_t lab = W.L.lab[i];
    uint32_t bm = W.L.bmask[i];
    uint32_t dlo = 0, dhi = 0, dlen = 0xFFFFFFFFu;
    int nchk = 0;
    while (bm) {
        const int b = __ffs(bm) - 1;
        bm &= bm - 1;
        uint32_t lo, hi;
        if (W.sc_v[i][b] == W.t[b]) {
            lo = W.sc_lo[i][b];
            hi = W.sc_hi[i][b];
        } else {
            find_slice(G, W.t[b], lab, (W.L.bdir[i] >> (2 * b)) & 3u, lo, hi, bytes);
            if (lane == 0) {
                W.sc_lo[i][b] = lo;
                W.sc_hi[i][b] = hi;
                W.sc_v[i][b] = W.t[b];
            }
        }
        if (lo == hi) return false;
        const uint32_t len = hi - lo;
        if (len < dlen) {
            if (dlen != 0xFFFFFFFFu) {
                if (lane == 0) { W.clo[i][nchk] = dlo; W.chi[i][nchk] = dhi; }
                nchk++;
            }
            dlo = lo; dhi = hi; dlen = len;
        } else {
            if (lane == 0) { W.clo[i][nchk] = lo; W.chi[i][nchk] = hi; }
            nchk++;
        }
    }
    if (lane == 0) { W.lo[i] = dlo; W.hi[i] = dhi; W.nchk[i] = nchk; }
    __syncwarp();
    return true;
}

// Static one-hop filter: a data vertex can host a pattern vertex only if its degree is at least
// the pattern vertex's and every label the pattern vertex's neighbours carry (ranks < 64) occurs
// among its own neighbours.  Depends on the data vertex alone, so it rejects only vertices that
// belong to no map at all.
__device__ __forceinline__ bool vertex_fits(const DevGraphView &G, int32_t c, uint32_t deg_req,
                                            unsigned long long need) {
    const VRec *r = G.vrec + c;
    const uint32_t deg = __ldg(&r->deg);
    const unsigned long long have = __ldg(reinterpret_cast<const unsigned long long *>(&r->nbr_labels));
    return deg >= deg_req && (have & need) == need;
}

// Candidate test at level i.  rej collects the earlier levels whose bound vertex caused a
// rejection by injectivity (the conflict set of conflict-directed backjumping).
__device__ __forceinline__ bool check_candidate(const DevGraphView &G, const WarpState &W, int i,
                                                int32_t c, const uint32_t *used,
                                                uint32_t &probes, uint32_t &rej) {
    uint32_t im = W.L.injmask[i];
    while (im) {
        const int b = __ffs(im) - 1;
        im &= im - 1;
        if (W.t[b] == c) { rej |= 1u << b; return false; }
    }
    if (used) {
        probes++;
        if (used_bit(used, c)) return false;
    }
    probes += 4;
    if (!vertex_fits(G, c, W.L.deg[i], W.need[W.L.vert[i]])) return false;
    const int nchk = W.nchk[i];
    for (int k = 0; k < nchk; k++)
        if (!contains(G.adj, W.clo[i][k], W.chi[i][k], c, probes)) return false;
    return true;
}

// Lexicographically first map (in the level order of W.L) with level 0 bound to `root` and no
// vertex in `used` (nullable).  On success W.t holds the map by level.
//
// Depth-first search with conflict-directed backjumping (Prosser, Computational Intelligence
// 9(3), 1993): when every candidate of level i has failed, the search returns directly to the
// deepest earlier level whose binding could change that outcome -- the levels that define
// level i's candidate slices (its pattern neighbours), the levels whose vertex rejected a
// candidate by injectivity, and the conflict levels handed up by deeper failures.  Levels in
// between cannot make level i succeed, so skipping their remaining candidates removes only
// subtrees without a map: the first map found in lexicographic order is unchanged.
//
// Resumable: with budget > 0 the search stops after `budget` candidate chunks and returns
// DFS_SUSPENDED with its whole state in W (current level in W.level).  It may later continue
// (resume = true) under a larger used set: bound vertices that have become used are dropped
// (the search continues at the first such level with that level's remaining candidates) and
// every popped candidate is re-tested against the used set.  Everything skipped before the
// suspension failed under the smaller used set and fails under the larger one, so the first map
// found is the first map avoiding the current used set.
enum : int { DFS_NONE = 0, DFS_FOUND = 1, DFS_SUSPENDED = 2, DFS_NOROOM = 3 };

// Counters of the search's algorithmic work (warp-uniform): driver-slice entries scanned, and
// partial maps bound, each weighted by its length (level + 1).
struct SearchWork {
    uint32_t scanned = 0, bound = 0;  // per search: at most budget x 32 entries
};

// Drain: once most warps of a search launch have run out of work items, the searches still
// running suspend at their next check (every DRAIN_EVERY chunks, after DRAIN_MIN_STEPS) instead
// of running to the round's budget, so the launch ends and the next round starts; a suspended
// search resumes (and may be split) there.  Suspension points never change a result.
constexpr uint32_t DRAIN_EVERY = 16;
constexpr uint32_t DRAIN_MIN_STEPS = 32;

__device__ __forceinline__ bool drain_requested(const int32_t *drain) {
    int d = 0;
    if ((threadIdx.x & 31) == 0) d = *reinterpret_cast<const volatile int32_t *>(drain);
    return __shfl_sync(FULLMASK, d, 0) != 0;
}

__device__ inline int dfs_run(const DevGraphView &G, WarpState &W, const uint32_t *used, int32_t root,
                       unsigned long long &bytes, uint32_t &probes, uint32_t &steps, uint32_t budget,
                       bool resume, SearchWork &work, const int32_t *drain = nullptr) {
    const int lane = threadIdx.x & 31;
    const int n = W.n;
    int i = 1;
    bool ok;
    uint32_t hi = 0, pos = 0, base = 0, mask = 0, conf = 0;
    if (!resume) {
        if (lane == 0) { W.t[0] = root; W.floor = 1; }
        __syncwarp();
        if (used) {
            bytes += 4;
            if (used_bit(used, root)) return DFS_NONE;
        }
        bytes += 32;
        if (!vertex_fits(G, root, W.L.deg[0], W.need[W.L.vert[0]])) return DFS_NONE;
        ok = enter_level(G, W, 1, bytes);
        if (ok) { hi = W.hi[1]; pos = W.lo[1]; }
    } else {
        if (used && used_bit(used, W.t[0])) return DFS_NONE;
        i = W.level;
        for (int l = 1; l < i; l++)
            if (used && used_bit(used, W.t[l])) {
                if (l < W.floor) return DFS_NONE;  // a binding this sub-search may not change
                i = l;
                break;
            }
        hi = W.hi[i]; pos = W.pos[i]; base = W.base[i]; mask = W.mask[i]; conf = W.conf[i];
        ok = true;
    }
    for (;;) {
        if (!ok) {
            // level i has no candidate left: jump to the deepest level of its conflict set;
            // below the floor the search space of this (sub-)search is exhausted
            const uint32_t cs = (conf | W.L.bmask[i]) & ((1u << i) - 1u);
            const int h = 31 - __clz(cs);
            if (h < W.floor) return DFS_NONE;
            conf = W.conf[h] | (cs & ~(1u << h));
            i = h;
            hi = W.hi[i]; pos = W.pos[i]; base = W.base[i]; mask = W.mask[i];
            ok = true;
            continue;
        }
        if (mask == 0) {
            if (pos >= hi) { ok = false; continue; }
            if (budget && (steps >= budget || (drain && steps >= DRAIN_MIN_STEPS && steps % DRAIN_EVERY == 0 &&
                                               drain_requested(drain)))) {
                if (lane == 0) {
                    W.level = i;
                    W.hi[i] = hi; W.pos[i] = pos; W.base[i] = base; W.mask[i] = 0; W.conf[i] = conf;
                }
                __syncwarp();
                return DFS_SUSPENDED;
            }
            const uint32_t k = pos + lane;
            bool good = false;
            uint32_t rej = 0;
            if (k < hi) good = check_candidate(G, W, i, __ldg(G.adj + k), used, probes, rej);
            mask = __ballot_sync(FULLMASK, good);
            conf |= __reduce_or_sync(FULLMASK, rej);
            work.scanned += min(32u, hi - pos);  // slice entries scanned: 4 bytes each in the algorithmic bytes
            steps++;
            base = pos;
            pos += 32;
            continue;
        }
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        const int32_t c = __ldg(G.adj + base + j);
        if (resume && used && used_bit(used, c)) continue;  // became used since the chunk scan
        if (lane == 0) W.t[i] = c;
        work.bound += (unsigned)(i + 1);
        if (i == n - 1) {  // keep the position so that a later resume continues past this map
            if (lane == 0) { W.level = i; W.hi[i] = hi; W.pos[i] = pos; W.base[i] = base; W.mask[i] = mask; W.conf[i] = conf; }
            __syncwarp();
            return DFS_FOUND;
        }
        if (lane == 0) { W.pos[i] = pos; W.base[i] = base; W.mask[i] = mask; W.conf[i] = conf; }
        __syncwarp();
        ++i;
        conf = 0;
        ok = enter_level(G, W, i, bytes);
        if (ok) { hi = W.hi[i]; pos = W.lo[i]; mask = 0; }
    }
}


__device__ __forceinline__ void load_level_plan(WarpState &W, const LevelPlan &L, const Plan &P) {
    const int lane = threadIdx.x & 31;
    constexpr int WORDS = sizeof(LevelPlan) / 4;
    if (lane < WORDS) reinterpret_cast<uint32_t *>(&W.L)[lane] = reinterpret_cast<const uint32_t *>(&L)[lane];
    if (lane < MAXN) W.need[lane] = P.need[lane];
    if (lane == 0) W.n = P.n;
    // a new plan: no cached slice is valid
    for (int k = lane; k < MAXN * MAXN; k += 32) (&W.sc_v[0][0])[k] = -1;
    __syncwarp();
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
    return v;
}

// Block-wide exclusive scan of one int per thread; returns the total.
__device__ __forceinline__ int block_scan(int v, int &excl, int *sh /* >= 33 ints */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULLMASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULLMASK, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sh[lane] = t;  // inclusive prefix of warp totals
        if (lane == nw - 1) sh[32] = t;
    }
    __syncthreads();
    excl = x - v + (w > 0 ? sh[w - 1] : 0);
    const int total = sh[32];
    __syncthreads();
    return total;
}

#define CK(x)                                                                         \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) {                                                      \
            fprintf(stderr, "flexis: %s failed: %s\n", #x, cudaGetErrorString(e_));  \
            return e_ == cudaErrorMemoryAllocation ? FLEXIS_E_NOMEM : FLEXIS_E_CUDA;  \
        }                                                                             \
    } while (0)

struct PatState;
struct Ctl;
struct EnumWS;

// Evaluation workspace: P pattern slots with their used bitmaps, windows and work items.
struct Workspace {
    int32_t P = 0;           // pattern capacity
    int64_t slots = 0;       // window-slot capacity (patterns x window size)
    int64_t sel_slots = 0;   // selection-log capacity (patterns x maps)
    int64_t bytes = 0;       // device bytes held
    PatState *st = nullptr;
    uint32_t *used = nullptr;
    int32_t *dirty = nullptr;
    int32_t clean = 0;  // patterns [0, clean) have all-zero used bitmaps between evaluations
    int32_t *win_root = nullptr, *win_state = nullptr, *win_map = nullptr;
    int2 *items = nullptr;
    Ctl *ctl = nullptr;
    int32_t *sel_buf = nullptr;
    unsigned long long *mni_seg = nullptr;
    uint32_t *susp = nullptr;
    int32_t *alist = nullptr;
    Plan *plans = nullptr;                   // device plan array (host-plan entry points)
    flexis_support_result *results = nullptr;
    int32_t plans_cap = 0;
    Ctl *h_ctl = nullptr;                    // pinned
};

struct DeviceGraph {
    int device = 0;
    cudaStream_t stream = nullptr;
    DevGraphView view{};
    void *d_vrec = nullptr, *d_runs = nullptr, *d_adj = nullptr, *d_labvtx = nullptr;
    int64_t bytes = 0;
    int64_t upload_bytes = 0;  // host-to-device bytes of the load (layout arrays, or the edge list)
    int32_t built_on_device = 0;
    int64_t vrec_count = 0, runs_words = 0, adj_words = 0, labvtx_words = 0;  // allocated sizes
    int sm_count = 0, l2 = 0;
    Workspace ws;
    int32_t last_P = 0, last_sel = 0;
    cudaEvent_t ev[2]{};
    std::vector<cudaEvent_t> sev;
    cudaGraphExec_t round_exec = nullptr;  // the captured round loop of the last level
    std::vector<cudaEvent_t> gev;          // search-launch events inside the captured graph
    int64_t graph_instantiations = 0, graph_fallbacks = 0;
    int commit_small_blocks = 0;  // one wave of the small-horizon commit kernel
    int32_t max_degree = 0;
    EnumWS *ews = nullptr;        // map enumerator workspace (enumerate.cu), allocated on first use
};

// Map enumerator (enumerate.cu): counts every map of the plans that ask for it into their
// results' n_maps (and materialises maps for the exact MIS); runs on `stream` after the greedy
// phase.  A deadline (measured from t_start) marks unfinished counts FLEXIS_E_TIMEOUT.
int dev_enumerate(DeviceGraph *g, const Plan *d_plans, int32_t P, flexis_support_result *d_results,
                  cudaStream_t stream, const EvalConfig &cfg, flexis_stats *stats,
                  std::chrono::steady_clock::time_point t_start);
void enum_ws_destroy(DeviceGraph *g);

// Exclusive prefix sum of cnt_off[0, n) in place, cnt_off[n] set to the total (enumerate.cu).
// tsum: scratch of scan_tsum_len(n) words.  Three launches on s.
constexpr int SCAN_TILE = 2048;  // elements per block of the scan (1024 threads x 2)
inline long long scan_tsum_len(long long n) { return n / SCAN_TILE + 2; }
int dev_scan_u64(unsigned long long *cnt_off, long long n, unsigned long long *tsum, cudaStream_t s);

// The object, stream, events and kernel attributes of a device graph, with no arrays (kernels.cu).
int dev_graph_init(int device, DeviceGraph **out);

}  // namespace fx
