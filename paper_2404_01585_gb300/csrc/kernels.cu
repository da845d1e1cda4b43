// sm_103a kernels of the FLEXIS support-evaluation path and the batched driver.
//
// What is computed (per pattern, all integer):
//   mIS  : the greedy maximal independent set of the pattern's maps (Sec. 2.4.3) taken in the
//          fixed order (H(seed, root), root, lexicographic tuple in matching order): roots are
//          visited in hash order (or by vertex id, the root-order variant; the order lives only
//          in the root index built at load), each root selects its lexicographically first map that
//          avoids vertices already used and then stops (Sec. 3.2.2, changes 1 and 2).  EARLY
//          mode stops at c = max(tau, 1) selections (Sec. 3.1.1).
//   MNI  : min over automorphism orbits of the number of distinct data vertices that some map
//          sends the orbit's vertices to (Sec. 2.4.4).
//   tau / frequent (Eq. tau).
//
// How the sequential greedy is made parallel without changing its result (speculation by
// windows, per pattern):
//   * a window holds the next W roots in greedy order; every root in it needing a map gets one
//     warp that searches its lexicographically first map avoiding the *current* used set
//     (k_search, warp-cooperative depth-first search over label slices);
//   * k_commit builds, in shared memory, an inverted index vertex -> smallest window slot whose
//     map holds it (the owner), finds the first slot f whose map shares a vertex with an
//     earlier slot's map, and commits every slot before f: each of those maps is the first map
//     of its root avoiding the vertices of all earlier selections, exactly as in the sequential
//     greedy.  Slots after f keep their maps unless a committed map took one of their vertices
//     (a map that avoids a smaller used set and also avoids the larger one is still the first
//     one: used sets only grow).  Roots without a map are decided at once for the same reason.
//   * new roots refill the window; the loop ends when c maps are selected or the roots run out.
// The result is therefore bit-identical to the sequential greedy for any window size, launch
// shape or batch composition.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "fx_kern.cuh"

namespace fx {

// window slot states.  A SEQ slot's root search ran out of its per-round budget: its remaining
// search space is an ordered list of saved sub-searches (the first one's index in the slot's
// map entry 0, each saved state holding the index of the next); the slot's map is the map of
// the first sub-search in that order that finds one, once every earlier one has found none.
enum : int32_t { SLOT_NEEDS = 0, SLOT_MAP = 1, SLOT_NONE = 2, SLOT_SEQ = 3 };
// saved sub-search status (word SUSP_STATUS of its saved state); its map in SUSP_MAP..+7
enum : int32_t { SS_PENDING = 0, SS_NONE = 1, SS_FOUND = 2 };
constexpr int SPLIT_MAX = 15;  // pieces one split may create


// slot phases: free, greedy rounds, MNI pending, result ready
enum : int32_t { PH_FREE = 0, PH_GREEDY = 1, PH_MNI = 2, PH_READY = 3 };

struct PatState {
    int64_t count;     // maps selected so far
    int64_t searched;  // root searches run
    int32_t cursor;    // next root (index into lab_vtx)
    int32_t nwin;      // slots in the window
    int32_t W;         // target window size
    int32_t done;
    int32_t exhausted; // every root processed
    int32_t rounds;
    int32_t phase;
    int32_t logged;    // selected maps written to the selection log
    unsigned long long mni_cnt[MAXN];
    unsigned long long steps;  // candidate chunks scanned by the greedy searches
    uint32_t max_steps;        // largest chunk count of one greedy search
    int32_t buf;               // current window buffer (0 or 1)
    uint32_t susp_mask;        // saved-search slots in use (KSUSP bits)
    uint32_t cancelled;        // stopped at a deadline before its decision
    uint32_t mni_cut;          // the MNI pass passed the deadline before this pattern's count
    int32_t ndirty;            // used-bitmap words this pattern made non-zero (listed up to DIRTY_CAP)
};

struct Ctl {
    int32_t n_items[2];
    int32_t next_item[2];
    int32_t active[2];
    int32_t acount[2];    // lengths of the two active-pattern lists
    int32_t idle[2];      // warps of the search launch that found no work item left
    int32_t drain[2];     // set once idle reaches the launch's drain threshold
    int32_t err;
    int32_t pad;
    unsigned long long bytes_greedy;
    unsigned long long bytes_mni;
    unsigned long long alg_scanned;   // greedy search: driver-slice entries scanned (A)
    unsigned long long alg_bound;     // greedy search: sum over bound partial maps of their length
    unsigned long long alg_map_words; // greedy search: words of the maps it wrote (n per map found)
    unsigned long long search_items;
    unsigned long long mni_items;
    unsigned long long mni_total;
    unsigned long long mni_next;
    unsigned long long t0_ns;     // device clock at the start of the evaluation (k_init)
};

struct Batch {
    DevGraphView G;
    const Plan *plans;
    int32_t P;
    int32_t Wmax;
    int32_t Wmin;
    int32_t sel_cap;
    uint32_t budget;      // per-round candidate chunks of one root search (0: unlimited)
    int32_t split_max;    // pieces per split (0: no split)
    uint32_t sid_all;     // saved sub-search indices a pattern may use (bit set)
    PatState *st;
    uint32_t *used;       // [P][words]
    int32_t *dirty;       // [P][DIRTY_CAP] words of `used` made non-zero (nullable: not tracked)
    int32_t *win_root;    // [P][2][Wmax]  two window buffers per pattern
    int32_t *win_state;   // [P][2][Wmax]
    int32_t *win_map;     // [P][2][Wmax][8] (by level)
    int2 *items;          // [P*Wmax] (pattern, buffer * Wmax + slot)
    Ctl *ctl;
    int32_t *sel;         // [P][sel_cap][8] selected maps, canonical vertex order
    unsigned long long *mni_seg;  // [P*8+1] prefix sums of MNI candidate segments
    int32_t *alist;               // [2][P] patterns still in their greedy phase (nullable: all)
    uint32_t *susp;               // [P][KSUSP][DFS_SAVE_STRIDE] saved search states
    flexis_support_result *results;
    unsigned long long deadline_ns;  // > 0: the MNI pass stops this long after ctl->t0_ns
};

// The device's global nanosecond clock (PTX special register %globaltimer).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int DFS_SAVE_WORDS = (int)(offsetof(WarpState, need) / 4);
constexpr int DFS_SAVE_STRIDE = 192;  // words per saved sub-search
constexpr int SUSP_STATUS = DFS_SAVE_WORDS;      // SS_* of the saved sub-search
constexpr int SUSP_NEXT = DFS_SAVE_WORDS + 1;    // next sub-search of the same slot, or -1
constexpr int SUSP_MAP = DFS_SAVE_WORDS + 2;     // its map (by level) when SS_FOUND
static_assert(SUSP_MAP + MAXN <= DFS_SAVE_STRIDE, "saved search state too large");
constexpr int KSUSP = 32;             // saved sub-searches a pattern may hold at once
constexpr uint32_t SEARCH_BUDGET = 4096;  // candidate chunks a root search runs per round


// ------------------------------------------------------------------ kernels
constexpr int SEARCH_THREADS = 256;
constexpr int DRAIN_DIV = 8;  // the searches drain once all but 1/DRAIN_DIV of the launch's warps are idle
constexpr int DIRTY_CAP = 1024;  // listed used-bitmap words per pattern (4 KB)
constexpr int COMMIT_THREADS = 256;

__device__ void reset_ctl(Ctl *c) {
    c->n_items[0] = c->n_items[1] = 0;
    c->next_item[0] = c->next_item[1] = 0;
    c->active[0] = c->active[1] = 0;
    c->idle[0] = c->idle[1] = 0;
    c->drain[0] = c->drain[1] = 0;
    c->err = 0;
    c->bytes_greedy = c->bytes_mni = 0;
    c->alg_scanned = c->alg_bound = c->alg_map_words = 0;
    c->search_items = c->mni_items = 0;
    c->mni_total = c->mni_next = 0;
}

__device__ void init_slot(const Batch &B, int p) {
    const Plan &P = B.plans[p];
    PatState s;
    memset(&s, 0, sizeof s);
    s.cursor = P.root_begin;
    s.W = B.Wmin;
    const bool nothing = P.status != FLEXIS_OK || (P.flags & FLEXIS_FLAG_ABSENT_LABEL) ||
                         P.root_begin >= P.root_end || P.skip_mis;
    s.done = nothing ? 1 : 0;
    s.exhausted = nothing ? 1 : 0;
    s.phase = nothing ? PH_MNI : PH_GREEDY;
    B.st[p] = s;
}

// closed batch: every slot [0, P) starts (the control words are zeroed before the launch); with
// an active list, the patterns that have a greedy phase form list 0
__global__ void k_init(Batch B) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) B.ctl->t0_ns = global_ns();
    if (p >= B.P) return;
    init_slot(B, p);
    if (B.alist && B.st[p].phase == PH_GREEDY) B.alist[atomicAdd(&B.ctl->acount[0], 1)] = p;
}

// serving: (re)start the listed slots and clear their used bitmaps; one block per slot
__global__ void k_admit(Batch B, const int32_t *slots, int n) {
    if (blockIdx.x >= n) return;
    const int p = slots[blockIdx.x];
    uint32_t *u = B.used + (size_t)p * B.G.words;
    for (int w = threadIdx.x; w < B.G.words; w += blockDim.x) u[w] = 0;
    if (threadIdx.x == 0) init_slot(B, p);
}

__global__ void k_reset_ctl(Batch B) { reset_ctl(B.ctl); }

// Claim up to `want` free saved-sub-search indices of a pattern; returns them as a bit set.
__device__ unsigned int claim_sids(unsigned int *m, int want, unsigned int ALL) {
    unsigned int cur = atomicAdd(m, 0u);
    for (int tries = 0; tries < 64; tries++) {
        unsigned int freeb = ~cur & ALL, take = 0;
        for (int k = 0; k < want && freeb; k++) {
            const unsigned int b = freeb & (~freeb + 1u);
            take |= b;
            freeb &= ~b;
        }
        if (!take) return 0;
        const unsigned int prev = atomicCAS(m, cur, cur | take);
        if (prev == cur) return take;
        cur = prev;
    }
    return 0;
}

__device__ __forceinline__ void save_state(uint32_t *dst, const WarpState &W, int status) {
    const int lane = threadIdx.x & 31;
    for (int w = lane; w < DFS_SAVE_WORDS; w += 32) dst[w] = reinterpret_cast<const uint32_t *>(&W)[w];
    if (lane == 0) dst[SUSP_STATUS] = status;
    if (status == SS_FOUND && lane < MAXN) dst[SUSP_MAP + lane] = W.t[lane];
    __syncwarp();
}

// One warp per work item.  Item (pattern, slot): a fresh search for the first map of the slot's
// root avoiding the used set.  Item (pattern, slot, saved sub-search): continue that sub-search.
// A search that uses up its per-round budget is saved; if it heads its slot it is also split:
// the unscanned candidates of its shallowest level with any left go to up to five new
// sub-searches, in order, and a continuation takes over everything after them.  Once all but an
// eighth of the launch's warps have found the item list empty, the searches still running are
// saved (and split) the same way at their next drain check instead of running to the budget,
// so a launch is not held open by a few long searches while most of the GPU idles.
__global__ void __launch_bounds__(SEARCH_THREADS, 6) k_search(Batch B, int q) {
    __shared__ WarpState ws[SEARCH_THREADS / 32];
    const int lane = threadIdx.x & 31;
    WarpState &W = ws[threadIdx.x >> 5];
    const int n_items = *reinterpret_cast<volatile int32_t *>(&B.ctl->n_items[q]);
    if (blockIdx.x == 0 && threadIdx.x == 0) B.ctl->acount[q] = 0;  // list q has been consumed
    if (lane == 0) W.acc_scanned = W.acc_bound = W.acc_maps = 0;
    for (;;) {
        SearchWork work;
        // the search's touched-bytes counts are not kept here (the algorithmic bytes are):
        // unused, the compiler drops them from the hot loop
        unsigned long long bytes = 0;
        uint32_t probes = 0;
        int it = 0;
        if (lane == 0) it = atomicAdd(&B.ctl->next_item[q], 1);
        it = __shfl_sync(FULLMASK, it, 0);
        if (it >= n_items) {
            // out of items: count this warp; past the threshold the running searches drain
            if (lane == 0) {
                const int nw = (int)(gridDim.x * (blockDim.x >> 5));
                if (atomicAdd(&B.ctl->idle[q], 1) + 1 >= nw - nw / DRAIN_DIV) B.ctl->drain[q] = 1;
            }
            break;
        }
        const int2 item = B.items[it];
        const int p = item.x;
        const int off = item.y & 0xFFFFFF;
        const int sid_in = (item.y >> 24) - 1;
        const Plan &P = B.plans[p];
        const size_t slot = (size_t)p * 2 * B.Wmax + off;
        int32_t *seq = B.win_map + slot * MAXN;
        const int32_t root = B.win_root[slot];
        const uint32_t *used = B.used + (size_t)p * B.G.words;
        uint32_t *sbase = B.susp + (size_t)p * KSUSP * DFS_SAVE_STRIDE;
        const bool resume = sid_in >= 0;
        load_level_plan(W, P.greedy, P);
        if (resume) {
            const uint32_t *src = sbase + (size_t)sid_in * DFS_SAVE_STRIDE;
            for (int w = lane; w < DFS_SAVE_WORDS; w += 32) reinterpret_cast<uint32_t *>(&W)[w] = src[w];
            __syncwarp();
        }
        uint32_t steps = 0;
        int r = dfs_run(B.G, W, used, root, bytes, probes, steps, B.budget, resume, work, &B.ctl->drain[q]);
        if (lane == 0) {
            W.acc_scanned += work.scanned;
            W.acc_bound += work.bound;
            if (r == DFS_FOUND) W.acc_maps += (unsigned)P.n;
        }
        int sidA = sid_in;
        if (r == DFS_SUSPENDED) {
            const bool head = !resume || seq[0] == sid_in;
            // split level: the shallowest level this search may still rebind that has unscanned
            // candidates (shallow candidates carry the largest subtrees)
            int m = -1;
            for (int l = W.floor; l <= W.level; l++)
                if (W.pos[l] < W.hi[l]) { m = l; break; }
            const int pieces = (head && m >= 0) ? (int)min(W.hi[m] - W.pos[m], (uint32_t)B.split_max) : 0;
            unsigned int got = 0;
            if (lane == 0) {
                const int want = (resume ? 0 : 1) + (pieces > 0 ? pieces + 1 : 0);
                got = want ? claim_sids(&B.st[p].susp_mask, want, B.sid_all) : 0u;
            }
            got = __shfl_sync(FULLMASK, got, 0);
            if (!resume) {
                if (!got) {
                    // no free saved-state slot: the slot stays NEEDS (undecided) and its search
                    // starts over next round, when earlier sub-searches have released slots
                    r = DFS_NOROOM;
                } else {
                    sidA = __ffs(got) - 1;
                    got &= got - 1;
                }
            }
            if (r == DFS_SUSPENDED) {
                const int np = __popc(got) >= 2 ? min(pieces, __popc(got) - 1) : 0;
                unsigned int keep = 0, g1 = got;  // sids of the split: np pieces + the continuation
                for (int k = 0; k < (np ? np + 1 : 0); k++) {
                    const unsigned int b = g1 & (~g1 + 1u);
                    keep |= b;
                    g1 &= ~b;
                }
                if (lane == 0 && (got & ~keep)) atomicAnd(&B.st[p].susp_mask, ~(got & ~keep));
                const int32_t old_next = resume ? (int32_t)sbase[(size_t)sidA * DFS_SAVE_STRIDE + SUSP_NEXT] : -1;
                int32_t link = sidA;  // last sub-search of the new chain so far
                if (np > 0) {
                    const uint32_t a = W.pos[m], b = W.hi[m], len = b - a;
                    const int lvl0 = W.level, floor0 = W.floor;
                    const uint32_t mask_m = W.mask[m], conf_m = W.conf[m];
                    unsigned int g2 = keep;
                    for (int j = 0; j <= np; j++) {
                        const int sid = __ffs(g2) - 1;
                        g2 &= g2 - 1;
                        if (lane == 0) {
                            W.level = m;
                            W.mask[m] = 0;
                            if (j < np) {  // piece j: candidates [a + len*j/np, a + len*(j+1)/np) of level m
                                W.floor = m;
                                W.pos[m] = a + (uint32_t)((uint64_t)len * j / np);
                                W.hi[m] = a + (uint32_t)((uint64_t)len * (j + 1) / np);
                                W.conf[m] = 0;
                            } else {  // continuation: level m exhausted, plain backtracking below it
                                W.floor = floor0;
                                W.pos[m] = b;
                                W.hi[m] = b;
                                W.conf[m] = (1u << m) - 1u;
                            }
                        }
                        __syncwarp();
                        save_state(sbase + (size_t)sid * DFS_SAVE_STRIDE, W, SS_PENDING);
                        if (lane == 0) sbase[(size_t)link * DFS_SAVE_STRIDE + SUSP_NEXT] = (uint32_t)sid;
                        link = sid;
                    }
                    if (lane == 0) {  // the head keeps what it had scanned of level m, nothing more
                        W.level = lvl0;
                        W.floor = m;
                        W.pos[m] = a;
                        W.hi[m] = a;
                        W.mask[m] = mask_m;
                        W.conf[m] = conf_m;
                    }
                    __syncwarp();
                }
                save_state(sbase + (size_t)sidA * DFS_SAVE_STRIDE, W, SS_PENDING);
                if (lane == 0) {
                    if (np == 0) sbase[(size_t)sidA * DFS_SAVE_STRIDE + SUSP_NEXT] = (uint32_t)old_next;
                    else sbase[(size_t)link * DFS_SAVE_STRIDE + SUSP_NEXT] = (uint32_t)old_next;
                    if (!resume) {
                        seq[0] = sidA;
                        B.win_state[slot] = SLOT_SEQ;
                    }
                }
                __syncwarp();
            }
        }
        if (lane == 0 && steps) {
            atomicAdd(&B.st[p].steps, (unsigned long long)steps);
            atomicMax(&B.st[p].max_steps, steps);
        }
        if (r == DFS_FOUND || r == DFS_NONE) {
            if (!resume) {
                if (lane == 0) B.win_state[slot] = r == DFS_FOUND ? SLOT_MAP : SLOT_NONE;
                if (r == DFS_FOUND && lane < P.n) seq[lane] = W.t[lane];
            } else {  // the state is kept so that the sub-search can go on past its map
                save_state(sbase + (size_t)sid_in * DFS_SAVE_STRIDE, W, r == DFS_FOUND ? SS_FOUND : SS_NONE);
            }
        }
        __syncwarp();
    }
    if (lane == 0 && W.acc_scanned) {
        // algorithmic bytes: 4 per slice entry scanned, 8 per bound vertex, 4 per map vertex
        atomicAdd(&B.ctl->bytes_greedy, 4ull * W.acc_scanned + 8ull * W.acc_bound + 4ull * W.acc_maps);
        atomicAdd(&B.ctl->alg_scanned, W.acc_scanned);
        atomicAdd(&B.ctl->alg_bound, W.acc_bound);
        atomicAdd(&B.ctl->alg_map_words, W.acc_maps);
    }
}


// Map slots one commit examines: bounds the shared-memory inverted index (the window itself
// can be larger; slots past the horizon are simply kept for the next round).
// A round commits at most KM maps of a pattern (the map slots before its horizon).  The inverted
// index of those maps lives in a shared-memory hash table of 2 * KM * MAXN entries (keys + values:
// 16 * KM * MAXN bytes).  Small batches, whose windows reach thousands of slots, use KMAP (64 KB
// per block); large batches, whose windows stay at <= 1024 slots and whose round cost is the
// per-pattern work of a million active patterns, use KMAP_SMALL (16 KB) in 128-thread blocks, so
// that about three times as many patterns are committed at once.
constexpr int KMAP = 512;
constexpr int KMAP_SMALL = 128;
constexpr int COMMIT_THREADS_SMALL = 128;
constexpr int SMALL_COMMIT_WMAX = 1024;
template <int KM>
__host__ __device__ constexpr int commit_hash() { return 2 * KM * MAXN; }  // power of two for KM a power of two

__device__ __forceinline__ uint32_t hslot(int32_t v, int logT) {
    return ((uint32_t)v * 0x9E3779B1u) >> (32 - logT);
}

// Commit of one pattern by one block: inverted index of the window's maps, prefix commit, refill,
// new items.  The window lives in two global buffers per pattern; the kept slots and the refill go
// to the other buffer, which becomes current for the next search.
template <int KM>
__device__ __forceinline__ void commit_one(const Batch &B, int q, int p, int32_t *smem) {
    int32_t *keys = smem, *vals = smem + commit_hash<KM>();
    __shared__ int sh_scan[40];
    __shared__ int s_f, s_newcur, s_horizon, s_base;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    PatState *S = B.st + p;
    if (S->phase != PH_GREEDY) return;
    const Plan &P = B.plans[p];
    const int n = P.n;
    const int nwin = S->nwin;
    const int Wmax = B.Wmax;
    const int cur = S->buf, nxt = cur ^ 1;
    const size_t pb = (size_t)p * 2 * Wmax;
    const size_t cb = pb + (size_t)cur * Wmax, nb = pb + (size_t)nxt * Wmax;
    const int32_t *st_cur = B.win_state + cb, *rt_cur = B.win_root + cb, *mp_cur = B.win_map + cb * MAXN;
    int32_t *st_nxt = B.win_state + nb, *rt_nxt = B.win_root + nb, *mp_nxt = B.win_map + nb * MAXN;
    uint32_t *used = B.used + (size_t)p * B.G.words;
    uint32_t *sbase = B.susp + (size_t)p * KSUSP * DFS_SAVE_STRIDE;

    // 0. sub-search sequences: drop sub-searches that found nothing; a slot whose first
    //    remaining sub-search found a map takes that map (if a vertex of it has been used since,
    //    the sub-search goes on from there instead); a slot with none left has no map
    for (int s = tid; s < nwin; s += nthr) {
        if (st_cur[s] != SLOT_SEQ) continue;
        int32_t *sq = const_cast<int32_t *>(mp_cur) + (size_t)s * MAXN;
        int state = SLOT_SEQ;
        int32_t head = -1, last = -1;
        unsigned int release = 0;
        int32_t cur_sid = sq[0];
        for (int guard = 0; cur_sid >= 0 && guard < KSUSP; guard++) {
            uint32_t *e = sbase + (size_t)cur_sid * DFS_SAVE_STRIDE;
            const int32_t next = (int32_t)e[SUSP_NEXT];
            int status = (int)e[SUSP_STATUS];
            if (status == SS_FOUND && head < 0) {
                bool stale = false;
                for (int l = 0; l < n; l++) stale |= used_bit(used, (int32_t)e[SUSP_MAP + l]);
                if (stale) {
                    e[SUSP_STATUS] = SS_PENDING;
                    status = SS_PENDING;
                } else {
                    release |= 1u << cur_sid;  // this and every later sub-search are done with
                    for (int32_t r2 = next, g2 = 0; r2 >= 0 && g2 < KSUSP; g2++) {
                        release |= 1u << r2;
                        r2 = (int32_t)sbase[(size_t)r2 * DFS_SAVE_STRIDE + SUSP_NEXT];
                    }
                    for (int l = 0; l < n; l++) sq[l] = (int32_t)e[SUSP_MAP + l];
                    state = SLOT_MAP;
                    break;
                }
            }
            if (status == SS_NONE) {
                release |= 1u << cur_sid;
            } else {
                if (head < 0) head = cur_sid;
                else sbase[(size_t)last * DFS_SAVE_STRIDE + SUSP_NEXT] = (uint32_t)cur_sid;
                last = cur_sid;
            }
            cur_sid = next;
        }
        if (state == SLOT_SEQ) {
            if (head < 0) {
                state = SLOT_NONE;
            } else {
                sbase[(size_t)last * DFS_SAVE_STRIDE + SUSP_NEXT] = 0xFFFFFFFFu;
                sq[0] = head;
            }
        }
        if (release) atomicAnd(&S->susp_mask, ~release);
        const_cast<int32_t *>(st_cur)[s] = state;
    }
    __syncthreads();

    // 1. horizon: index of the (KM+1)-th map slot (or the window end)
    if (tid == 0) s_horizon = nwin;
    __syncthreads();
    int nmap = 0;
    for (int b0 = 0; b0 < nwin; b0 += nthr) {
        const int s = b0 + tid;
        const int ism = (s < nwin && st_cur[s] == SLOT_MAP) ? 1 : 0;
        int excl;
        const int tot = block_scan(ism, excl, sh_scan);
        if (ism && nmap + excl == KM) s_horizon = s;
        nmap += tot;
    }
    __syncthreads();
    const int horizon = s_horizon;
    const int nins = min(nmap, KM) * n;
    int logT = 6;
    while ((1 << logT) < 2 * nins) logT++;
    const int T = 1 << logT;
    for (int k = tid; k < T; k += nthr) { keys[k] = -1; vals[k] = INT_MAX; }
    if (tid == 0) s_f = horizon;
    __syncthreads();
    // 2. inverted index: vertex -> owner (smallest slot before the horizon whose map holds it)
    for (int idx = tid; idx < horizon * n; idx += nthr) {
        const int s = idx / n, k = idx - s * n;
        if (st_cur[s] != SLOT_MAP) continue;
        const int32_t v = mp_cur[(size_t)s * MAXN + k];
        uint32_t h = hslot(v, logT);
        for (;;) {
            const int32_t prev = atomicCAS(&keys[h], -1, v);
            if (prev == -1 || prev == v) { atomicMin(&vals[h], s); break; }
            h = (h + 1) & (T - 1);
        }
    }
    __syncthreads();
    auto owner = [&](int32_t v) -> int {  // INT_MAX when v is in no indexed map
        uint32_t h = hslot(v, logT);
        for (;;) {
            const int32_t k = keys[h];
            if (k == v) return vals[h];
            if (k == -1) return INT_MAX;
            h = (h + 1) & (T - 1);
        }
    };
    // 3. first slot whose map meets an earlier slot's map
    for (int idx = tid; idx < horizon * n; idx += nthr) {
        const int s = idx / n, k = idx - s * n;
        if (st_cur[s] != SLOT_MAP) continue;
        if (owner(mp_cur[(size_t)s * MAXN + k]) < s) atomicMin(&s_f, s);
    }
    // a suspended search, or one that found no room to be suspended and starts over, is
    // undecided: nothing at or after it can be committed yet
    for (int s = tid; s < horizon; s += nthr)
        if (st_cur[s] == SLOT_SEQ || st_cur[s] == SLOT_NEEDS) atomicMin(&s_f, s);
    __syncthreads();
    const int f = s_f;
    // 4. commit the map slots before f, in slot order
    const int64_t count0 = S->count;
    int ncommit = 0;
    for (int b0 = 0; b0 < f; b0 += nthr) {
        const int s = b0 + tid;
        const int isc = (s < f && st_cur[s] == SLOT_MAP) ? 1 : 0;
        int excl;
        const int tot = block_scan(isc, excl, sh_scan);
        if (isc) {
            const int32_t *m = mp_cur + (size_t)s * MAXN;
            for (int l = 0; l < n; l++) {
                const uint32_t wi = (uint32_t)m[l] >> 5;
                const uint32_t old = atomicOr(used + wi, 1u << (m[l] & 31));
                if (old == 0 && B.dirty) {  // first bit of this word: list it for the clean-up
                    const int k = atomicAdd(&S->ndirty, 1);
                    if (k < DIRTY_CAP) B.dirty[(size_t)p * DIRTY_CAP + k] = (int32_t)wi;
                }
            }
            const int64_t at = count0 + ncommit + excl;
            if (B.sel && at < B.sel_cap && at < P.cap) {
                int32_t *o = B.sel + ((size_t)p * B.sel_cap + at) * MAXN;
                for (int l = 0; l < n; l++) o[P.greedy.vert[l]] = m[l];
            }
        }
        ncommit += tot;
    }
    __syncthreads();  // the used bits of step 4 are read by the refill of step 7
    // 5. keep the slots from f on that still matter, in order, in the other buffer; a kept map
    //    needs a new search if a committed map took one of its vertices
    int keep_n = 0;
    for (int b0 = f; b0 < nwin; b0 += nthr) {
        const int s = b0 + tid;
        const int kp = (s < nwin && st_cur[s] != SLOT_NONE) ? 1 : 0;
        int excl;
        const int tot = block_scan(kp, excl, sh_scan);
        if (kp) {
            const int r = keep_n + excl;
            int state = st_cur[s];
            if (state == SLOT_MAP) {
                const int32_t *m = mp_cur + (size_t)s * MAXN;
                for (int l = 0; l < n; l++) {
                    mp_nxt[(size_t)r * MAXN + l] = m[l];
                    if (owner(m[l]) < f) state = SLOT_NEEDS;
                }
            } else if (state == SLOT_SEQ) {
                for (int l = 0; l < MAXN; l++) mp_nxt[(size_t)r * MAXN + l] = mp_cur[(size_t)s * MAXN + l];
            }
            rt_nxt[r] = rt_cur[s];
            st_nxt[r] = state;
        }
        keep_n += tot;
    }
    // 6. window size: grow while speculation is conflict-free
    int W = S->W;
    if (nwin > 0 && f >= nwin) W = min(2 * W, Wmax);
    // 7. refill from the root order; a used root, or one that cannot host canonical vertex 0,
    //    has no map and is decided on the spot
    int nw = keep_n;
    int cursor = S->cursor;
    const int rend = P.root_end;
    while (nw < W && cursor < rend) {
        const int chunk = min(nthr, rend - cursor);
        const int need = W - nw;
        int ok = 0;
        int32_t r = -1;
        if (tid < chunk) {
            r = __ldg(B.G.lab_vtx + cursor + tid);
            ok = (!used_bit(used, r) && vertex_fits(B.G, r, P.greedy.deg[0], P.need[0])) ? 1 : 0;
        }
        if (tid == 0) s_newcur = cursor + chunk;
        __syncthreads();
        int excl;
        const int tot = block_scan(ok, excl, sh_scan);
        if (ok && excl < need) {
            rt_nxt[nw + excl] = r;
            st_nxt[nw + excl] = SLOT_NEEDS;
            if (excl == need - 1) s_newcur = cursor + tid + 1;
        }
        __syncthreads();
        nw += min(tot, need);
        cursor = s_newcur;
        __syncthreads();
    }
    // 8. one search item for every slot that needs a map
    __syncthreads();
    // items: a fresh search per NEEDS slot, one continuation per pending sub-search of a SEQ slot
    auto n_items_of = [&](int s) -> int {
        if (s >= nw) return 0;
        const int st = st_nxt[s];
        if (st == SLOT_NEEDS) return 1;
        if (st != SLOT_SEQ) return 0;
        int c = 0;
        for (int32_t r2 = mp_nxt[(size_t)s * MAXN], g2 = 0; r2 >= 0 && g2 < KSUSP; g2++) {
            const uint32_t *e = sbase + (size_t)r2 * DFS_SAVE_STRIDE;
            c += (int)(e[SUSP_STATUS] == SS_PENDING);
            r2 = (int32_t)e[SUSP_NEXT];
        }
        return c;
    };
    int nitems = 0;
    for (int b0 = 0; b0 < nw; b0 += nthr) {
        int excl;
        nitems += block_scan(n_items_of(b0 + tid), excl, sh_scan);
    }
    if (tid == 0) s_base = nitems ? atomicAdd(&B.ctl->n_items[q], nitems) : 0;
    __syncthreads();
    int wr = s_base;
    for (int b0 = 0; b0 < nw; b0 += nthr) {
        const int s = b0 + tid;
        const int nd = n_items_of(s);
        int excl;
        const int tot = block_scan(nd, excl, sh_scan);
        if (nd) {
            const int o = nxt * Wmax + s;
            if (st_nxt[s] == SLOT_NEEDS) {
                B.items[wr + excl] = make_int2(p, o);
            } else {
                int w = wr + excl;
                for (int32_t r2 = mp_nxt[(size_t)s * MAXN], g2 = 0; r2 >= 0 && g2 < KSUSP; g2++) {
                    const uint32_t *e = sbase + (size_t)r2 * DFS_SAVE_STRIDE;
                    if (e[SUSP_STATUS] == SS_PENDING) B.items[w++] = make_int2(p, o | ((r2 + 1) << 24));
                    r2 = (int32_t)e[SUSP_NEXT];
                }
            }
        }
        wr += tot;
    }
    if (tid == 0) {
        const int64_t count = count0 + ncommit;
        S->count = count;
        if (B.sel) S->logged = (int32_t)min(min(count, P.cap), (int64_t)B.sel_cap);
        S->buf = nxt;
        S->cursor = cursor;
        S->nwin = nw;
        S->W = W;
        S->rounds++;
        S->searched += nitems;
        const bool reached = count >= P.cap;
        // every selection to come needs a root of its own: the roots in the window and those not
        // yet visited bound it; below c the pattern is infrequent, which is all mining asks
        const bool hopeless = P.decide_only && count + nw + (int64_t)(rend - cursor) < P.cap;
        const bool exhausted = (nw == 0 && cursor >= rend) || hopeless;
        if (reached || exhausted) {
            S->done = 1;
            S->exhausted = exhausted && !reached;
            S->phase = PH_MNI;
        } else {
            atomicAdd(&B.ctl->active[q], 1);
            if (B.alist) B.alist[(size_t)(q ^ 1) * B.P + atomicAdd(&B.ctl->acount[q ^ 1], 1)] = p;
        }
        if (nitems) atomicAdd(&B.ctl->search_items, (unsigned long long)nitems);
    }
}

// Dense form: one block per pattern slot.  Listed form: blocks walk the list of patterns still in
// their greedy phase (so late rounds of a large batch launch no block per finished pattern), and
// append the patterns that stay active to the other list.
template <int KM>
__global__ void __launch_bounds__(COMMIT_THREADS) k_commit(Batch B, int q) {
    extern __shared__ int32_t smem[];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        B.ctl->n_items[q ^ 1] = 0;
        B.ctl->next_item[q ^ 1] = 0;
        B.ctl->active[q ^ 1] = 0;
        B.ctl->idle[q ^ 1] = 0;
        B.ctl->drain[q ^ 1] = 0;
    }
    if (!B.alist) {
        commit_one<KM>(B, q, blockIdx.x, smem);
        return;
    }
    const int count = *reinterpret_cast<volatile int32_t *>(&B.ctl->acount[q]);
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        commit_one<KM>(B, q, B.alist[(size_t)q * B.P + i], smem);
        __syncthreads();
    }
}

// MNI segments: for every pattern whose mIS stayed below c and is not zero, one segment per
// orbit covering the orbit label's vertices.
__global__ void k_mni_setup(Batch B) {
    __shared__ int sh[40];
    __shared__ unsigned long long carry;
    const int tid = threadIdx.x;
    const int nseg = B.P * MAXN;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nseg; base += blockDim.x) {
        const int sidx = base + tid;
        int len = 0;
        if (sidx < nseg) {
            const int p = sidx / MAXN, o = sidx % MAXN;
            const Plan &P = B.plans[p];
            const PatState &S = B.st[p];
            // without a greedy phase nothing is known about the MNI: every orbit is searched
            const bool need = S.phase == PH_MNI && !S.cancelled && P.status == FLEXIS_OK && P.want_mni &&
                              !(P.flags & FLEXIS_FLAG_ABSENT_LABEL) &&
                              (P.skip_mis || (S.count < P.cap && S.count > 0));
            if (need && o < P.n_orb) {
                const int u = P.orb[o].vert[0];
                len = P.lab_end[u] - P.lab_begin[u];
            }
        }
        int excl;
        const int tot = block_scan(len, excl, sh);
        if (sidx < nseg) B.mni_seg[sidx] = carry + (unsigned long long)excl;
        __syncthreads();
        if (tid == 0) carry += (unsigned long long)tot;
        __syncthreads();
    }
    if (tid == 0) {
        B.mni_seg[nseg] = carry;
        B.ctl->mni_total = carry;
        B.ctl->mni_next = 0;
    }
}

constexpr int MNI_CHUNK = 8;
constexpr uint32_t MNI_BUDGET = 4096;  // candidate chunks of an MNI search between deadline checks

// One warp per candidate vertex d of an orbit: does some map send the orbit representative to d?
__global__ void __launch_bounds__(SEARCH_THREADS) k_mni(Batch B) {
    __shared__ WarpState ws[SEARCH_THREADS / 32];
    const int lane = threadIdx.x & 31;
    WarpState &W = ws[threadIdx.x >> 5];
    const unsigned long long total = *reinterpret_cast<volatile unsigned long long *>(&B.ctl->mni_total);
    const int nseg = B.P * MAXN;
    unsigned long long bytes = 0, items = 0, scanned_all = 0;
    uint32_t probes = 0;
    int cur_seg = -1;
    for (;;) {
        unsigned long long c0 = 0;
        if (lane == 0) c0 = atomicAdd(&B.ctl->mni_next, (unsigned long long)MNI_CHUNK);
        c0 = __shfl_sync(FULLMASK, c0, 0);
        if (c0 >= total) break;
        const unsigned long long c1 = min(total, c0 + MNI_CHUNK);
        for (unsigned long long c = c0; c < c1; c++) {
            // segment holding c: last seg with mni_seg[seg] <= c (and non-empty)
            int lo = 0, hi = nseg;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (B.mni_seg[mid] <= c) lo = mid; else hi = mid;
            }
            const int seg = lo;
            const int p = seg / MAXN, o = seg % MAXN;
            const Plan &P = B.plans[p];
            unsigned long long *cnt = &B.st[p].mni_cnt[o];
            if ((long long)__ldcg(cnt) >= P.cap) continue;
            if (seg != cur_seg) {
                load_level_plan(W, P.orb[o], P);
                cur_seg = seg;
            }
            const int u = P.orb[o].vert[0];
            const int32_t d = __ldg(B.G.lab_vtx + P.lab_begin[u] + (int)(c - B.mni_seg[seg]));
            items++;
            uint32_t steps = 0;
            // existence search in slices of MNI_BUDGET candidate chunks; between slices the
            // deadline is checked and the search resumes where it stopped
            SearchWork work;
            int r = dfs_run(B.G, W, nullptr, d, bytes, probes, steps, MNI_BUDGET, false, work);
            while (r == DFS_SUSPENDED) {
                if (B.deadline_ns && global_ns() - B.ctl->t0_ns > B.deadline_ns) {
                    if (lane == 0) B.st[p].mni_cut = 1u;
                    break;
                }
                steps = 0;
                r = dfs_run(B.G, W, nullptr, d, bytes, probes, steps, MNI_BUDGET, true, work);
            }
            scanned_all += work.scanned;
            if (r == DFS_FOUND && lane == 0) atomicAdd(cnt, 1ull);
        }
    }
    unsigned long long tot = warp_sum((unsigned long long)probes * 4ull) + (lane == 0 ? bytes + 4ull * scanned_all : 0ull);
    if (lane == 0) {
        if (tot) atomicAdd(&B.ctl->bytes_mni, tot);
        if (items) atomicAdd(&B.ctl->mni_items, items);
    }
}

// Deadline: patterns still in their greedy phase stop between two rounds (no search is in
// flight then) and are finalised with FLEXIS_E_TIMEOUT.  `slots` (nullable) lists the patterns
// to stop; NULL stops every pattern of the batch.
__global__ void k_cancel(Batch B, const int32_t *slots, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = slots ? slots[i] : i;
    PatState &S = B.st[p];
    if (S.phase != PH_GREEDY) return;
    S.cancelled = 1;
    S.done = 1;
    S.phase = PH_MNI;
}

// Leave every used bitmap of the batch zero again: a pattern that listed all the words it made
// non-zero clears those, one that overflowed its list clears its whole bitmap.  One warp per
// pattern.  The next evaluation then starts without clearing |V|/8 bytes per pattern.
__global__ void k_clear_used(Batch B) {
    const int p = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= B.P) return;
    uint32_t *u = B.used + (size_t)p * B.G.words;
    const int nd = B.st[p].ndirty;
    if (nd <= DIRTY_CAP) {
        const int32_t *d = B.dirty + (size_t)p * DIRTY_CAP;
        for (int i = lane; i < nd; i += 32) u[d[i]] = 0u;
    } else {
        for (uint32_t w = lane; w < B.G.words; w += 32) u[w] = 0u;
    }
}

__global__ void k_finalize(Batch B) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B.P) return;
    const Plan &P = B.plans[p];
    PatState &S = B.st[p];
    if (S.phase != PH_MNI) return;
    S.phase = PH_READY;
    flexis_support_result r;
    memset(&r, 0, sizeof r);
    r.status = P.status;
    r.n = P.n;
    r.sigma = P.sigma;
    r.tau = P.tau;
    r.cap = P.mode == FLEXIS_MODE_EARLY ? P.cap : -1;
    r.flags = P.flags;
    r.roots_searched = S.searched;
    r.search_steps = (int64_t)S.steps;
    r.max_item_steps = (int32_t)S.max_steps;
    r.rounds = S.rounds;
    r.mis_exact = -1;
    if (P.status == FLEXIS_OK) {
        const int64_t cap = P.cap;
        const int64_t mis = S.count < cap ? S.count : cap;
        int64_t mni;
        if (!P.want_mni) {
            mni = -1;
        } else if (P.flags & FLEXIS_FLAG_ABSENT_LABEL) {
            mni = 0;
        } else if (P.skip_mis) {
            mni = cap;
            for (int o = 0; o < P.n_orb; o++) mni = min(mni, min((int64_t)S.mni_cnt[o], cap));
            if (P.root_begin >= P.root_end) mni = 0;  // no root: M is empty
        } else if (S.count >= cap || S.count == 0) {
            mni = S.count >= cap ? cap : 0;
            r.flags |= FLEXIS_FLAG_MNI_FROM_MIS;
        } else {
            mni = cap;
            for (int o = 0; o < P.n_orb; o++) {
                const int64_t c = (int64_t)S.mni_cnt[o];
                mni = min(mni, min(c, cap));
            }
        }
        r.mis = mis;
        r.mni = mni;
        const int64_t c = P.tau > 1 ? P.tau : 1;
        r.frequent = mis >= c ? 1 : 0;
        if (P.mode == FLEXIS_MODE_EARLY) {
            if (S.count >= cap && !P.skip_mis) r.flags |= FLEXIS_FLAG_MIS_SATURATED;
            if (mni >= cap) r.flags |= FLEXIS_FLAG_MNI_SATURATED;
        }
        if (P.skip_mis) {
            r.mis = -1;
            r.frequent = 0;
        }
        if (S.cancelled) {
            // stopped before its decision: mis counts the maps committed so far (a lower bound
            // of the pattern's mIS); nothing is decided
            r.status = FLEXIS_E_TIMEOUT;
            r.mni = -1;
            r.frequent = 0;
        } else if (S.mni_cut && P.want_mni) {
            // the deadline passed during the MNI pass: mis and frequent are final, mni is not
            r.status = FLEXIS_E_TIMEOUT;
            r.mni = -1;
            r.flags &= ~(uint32_t)FLEXIS_FLAG_MNI_SATURATED;
        }
    }
    B.results[p] = r;
}

// ------------------------------------------------------------------ device graph + workspaces

template <class T>
static int upload(void **d, const std::vector<T> &h, cudaStream_t s, int64_t &bytes) {
    size_t b = std::max<size_t>(h.size(), 1) * sizeof(T);
    CK(cudaMalloc(d, b));
    CK(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    bytes += (int64_t)b;
    return FLEXIS_OK;
}

template <int KM>
static size_t commit_smem_of() { return sizeof(int32_t) * 2 * commit_hash<KM>(); }
static size_t commit_smem(int) { return commit_smem_of<KMAP>(); }

int dev_pattern_bytes(const DeviceGraph *g, int32_t Wmax, int32_t sel, int64_t *bytes) {
    *bytes = (int64_t)g->view.words * 4 + 4ll * DIRTY_CAP + (int64_t)Wmax * (2 * (4 + 4 + 4 * MAXN) + 8) + 8 * KSUSP +
             (int64_t)sizeof(PatState) + (int64_t)sizeof(Plan) + (int64_t)sizeof(flexis_support_result) +
             8 * (MAXN + 1) + (int64_t)sel * 4 * MAXN + 4ll * KSUSP * DFS_SAVE_STRIDE;
    return FLEXIS_OK;
}

int dev_free_bytes(const DeviceGraph *g, int64_t *bytes) {
    size_t fr = 0, tot = 0;
    CK(cudaSetDevice(g->device));
    CK(cudaMemGetInfo(&fr, &tot));
    *bytes = (int64_t)std::min(fr + (size_t)g->ws.bytes, tot);  // free + what the workspace holds
    return FLEXIS_OK;
}

int dev_graph_init(int device, DeviceGraph **out) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= device || device < 0) return FLEXIS_E_CUDA;
    DeviceGraph *g = new DeviceGraph();
    g->device = device;
    auto fail = [&](int code) { dev_graph_destroy(g); return code; };
    if (cudaSetDevice(device) != cudaSuccess) return fail(FLEXIS_E_CUDA);
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(FLEXIS_E_CUDA);
    if (cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->l2, cudaDevAttrL2CacheSize, device) != cudaSuccess ||
        cudaEventCreate(&g->ev[0]) != cudaSuccess || cudaEventCreate(&g->ev[1]) != cudaSuccess)
        return fail(FLEXIS_E_CUDA);
    if (cudaFuncSetAttribute(k_commit<KMAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)commit_smem_of<KMAP>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_commit<KMAP_SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)commit_smem_of<KMAP_SMALL>()) != cudaSuccess)
        return fail(FLEXIS_E_CUDA);
    {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_commit<KMAP_SMALL>, COMMIT_THREADS_SMALL,
                                                          commit_smem_of<KMAP_SMALL>()) != cudaSuccess)
            per_sm = 1;
        g->commit_small_blocks = g->sm_count * std::max(1, per_sm);
    }
    *out = g;
    return FLEXIS_OK;
}

int dev_graph_create(const HostGraph &hg, int device, DeviceGraph **out) {
    DeviceGraph *g = nullptr;
    int rc = dev_graph_init(device, &g);
    if (rc) return rc;
    auto fail = [&](int code) { dev_graph_destroy(g); return code; };
    if ((rc = upload(&g->d_vrec, hg.vrec, g->stream, g->bytes))) return fail(rc);
    if ((rc = upload(&g->d_runs, hg.runs, g->stream, g->bytes))) return fail(rc);
    if ((rc = upload(&g->d_adj, hg.adj, g->stream, g->bytes))) return fail(rc);
    if ((rc = upload(&g->d_labvtx, hg.lab_vtx, g->stream, g->bytes))) return fail(rc);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return fail(FLEXIS_E_CUDA);
    g->upload_bytes = g->bytes;
    g->vrec_count = (int64_t)std::max<size_t>(hg.vrec.size(), 1);
    g->runs_words = (int64_t)std::max<size_t>(hg.runs.size(), 1);
    g->adj_words = (int64_t)std::max<size_t>(hg.adj.size(), 1);
    g->labvtx_words = (int64_t)std::max<size_t>(hg.lab_vtx.size(), 1);
    g->view.vrec = (const VRec *)g->d_vrec;
    g->view.runs = (const uint32_t *)g->d_runs;
    g->view.adj = (const int32_t *)g->d_adj;
    g->view.lab_vtx = (const int32_t *)g->d_labvtx;
    g->view.nv = hg.nv;
    g->view.words = (int32_t)std::max<int64_t>(1, (hg.nv + 31) / 32);
    g->view.dstride = hg.directed ? hg.nv : 0;
    g->max_degree = hg.max_degree;
    *out = g;
    return FLEXIS_OK;
}

static void ws_free(Workspace &w) {
    cudaFree(w.st); cudaFree(w.used); cudaFree(w.dirty); cudaFree(w.win_root); cudaFree(w.win_state);
    cudaFree(w.win_map); cudaFree(w.items); cudaFree(w.ctl); cudaFree(w.sel_buf);
    cudaFree(w.mni_seg); cudaFree(w.plans); cudaFree(w.results); cudaFree(w.susp); cudaFree(w.alist);
    if (w.h_ctl) cudaFreeHost(w.h_ctl);
    w = Workspace();
}

// Capacity is kept in patterns and in window slots (patterns x Wmax) separately, so a large
// batch with small windows followed by a small batch with large windows never allocates the
// product of the two.
static int ws_ensure(const DeviceGraph *g, Workspace &w, int32_t P, int32_t Wmax, int32_t sel) {
    const int64_t slots = (int64_t)P * Wmax;
    if (P <= w.P && slots <= w.slots && (int64_t)P * sel <= w.sel_slots && w.h_ctl) return FLEXIS_OK;
    const int32_t nP = std::max(P, w.P);
    const int64_t nSlots = std::max(slots, w.slots);
    const int64_t nSel = std::max((int64_t)P * sel, w.sel_slots);
    ws_free(w);
    const size_t words = (size_t)g->view.words;
    int64_t b = 0;
    auto alloc = [&](void **ptr, size_t bytes) {
        b += (int64_t)bytes;
        return cudaMalloc(ptr, std::max<size_t>(bytes, 16));
    };
    CK(alloc((void **)&w.st, sizeof(PatState) * nP));
    CK(cudaMemset(w.st, 0, sizeof(PatState) * nP));
    CK(alloc((void **)&w.used, sizeof(uint32_t) * words * nP));
    CK(alloc((void **)&w.dirty, sizeof(int32_t) * (size_t)DIRTY_CAP * nP));
    w.clean = 0;
    CK(alloc((void **)&w.win_root, sizeof(int32_t) * (size_t)nSlots * 2));
    CK(alloc((void **)&w.win_state, sizeof(int32_t) * (size_t)nSlots * 2));
    CK(alloc((void **)&w.win_map, sizeof(int32_t) * (size_t)nSlots * 2 * MAXN));
    CK(alloc((void **)&w.items, sizeof(int2) * ((size_t)nSlots + (size_t)nP * KSUSP)));
    CK(alloc((void **)&w.ctl, sizeof(Ctl)));
    CK(alloc((void **)&w.mni_seg, sizeof(unsigned long long) * ((size_t)nP * MAXN + 1)));
    CK(alloc((void **)&w.susp, sizeof(uint32_t) * (size_t)nP * KSUSP * DFS_SAVE_STRIDE));
    CK(alloc((void **)&w.alist, sizeof(int32_t) * (size_t)nP * 2));
    CK(alloc((void **)&w.plans, sizeof(Plan) * (size_t)nP));
    CK(alloc((void **)&w.results, sizeof(flexis_support_result) * (size_t)nP));
    if (nSel > 0) CK(alloc((void **)&w.sel_buf, sizeof(int32_t) * (size_t)nSel * MAXN));
    CK(cudaMallocHost((void **)&w.h_ctl, sizeof(Ctl)));
    w.P = nP;
    w.slots = nSlots;
    w.sel_slots = nSel;
    w.bytes = b;
    return FLEXIS_OK;
}

void dev_graph_destroy(DeviceGraph *g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    ws_free(g->ws);
    enum_ws_destroy(g);
    cudaFree(g->d_vrec); cudaFree(g->d_runs); cudaFree(g->d_adj); cudaFree(g->d_labvtx);
    if (g->ev[0]) cudaEventDestroy(g->ev[0]);
    if (g->ev[1]) cudaEventDestroy(g->ev[1]);
    for (auto e : g->sev) cudaEventDestroy(e);
    if (g->round_exec) cudaGraphExecDestroy(g->round_exec);
    for (auto e : g->gev) cudaEventDestroy(e);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

int dev_graph_device(const DeviceGraph *g) { return g->device; }
int64_t dev_graph_bytes(const DeviceGraph *g) { return g->bytes; }

void dev_graph_load_info(const DeviceGraph *g, int64_t *upload_bytes, int32_t *on_device) {
    *upload_bytes = g->upload_bytes;
    *on_device = g->built_on_device;
}

int dev_graph_layout(const DeviceGraph *g, int32_t part, void *out, int64_t cap, int64_t *bytes) {
    const void *src = nullptr;
    int64_t size = 0;
    switch (part) {
        case 0: src = g->d_vrec; size = g->vrec_count * (int64_t)sizeof(VRec); break;
        case 1: src = g->d_runs; size = g->runs_words * 4; break;
        case 2: src = g->d_adj; size = g->adj_words * 4; break;
        case 3: src = g->d_labvtx; size = g->labvtx_words * 4; break;
        default: return FLEXIS_E_INVALID;
    }
    *bytes = size;
    if (!out) return FLEXIS_OK;
    if (cap < size) return FLEXIS_E_INVALID;
    CK(cudaSetDevice(g->device));
    CK(cudaMemcpyAsync(out, src, (size_t)size, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return FLEXIS_OK;
}
cudaStream_t dev_graph_stream(const DeviceGraph *g) { return g->stream; }
int dev_graph_props(const DeviceGraph *g, int *sm, int *l2) {
    *sm = g->sm_count;
    *l2 = g->l2;
    return FLEXIS_OK;
}

static Batch make_batch(const DeviceGraph *g, const Workspace &w, const Plan *plans, int32_t P,
                        int Wmin, int Wmax, int sel, flexis_support_result *results) {
    Batch B{};  // every field zero (null pointers) unless set below
    B.G = g->view;
    B.plans = plans;
    B.P = P;
    B.Wmax = Wmax;
    B.Wmin = Wmin;
    B.sel_cap = sel;
    B.budget = SEARCH_BUDGET;
    B.split_max = SPLIT_MAX;
    B.sid_all = KSUSP >= 32 ? 0xFFFFFFFFu : ((1u << (KSUSP & 31)) - 1u);
    B.st = w.st;
    B.used = w.used;
    B.dirty = w.dirty;
    B.win_root = w.win_root;
    B.win_state = w.win_state;
    B.win_map = w.win_map;
    B.items = w.items;
    B.ctl = w.ctl;
    B.sel = sel > 0 ? w.sel_buf : nullptr;
    B.mni_seg = w.mni_seg;
    B.susp = w.susp;
    B.alist = nullptr;  // dense: every slot of the batch is visited by the commit kernel
    B.results = results;
    return B;
}

static int search_grid(const DeviceGraph *g, const EvalConfig &cfg) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_search, SEARCH_THREADS, 0) != cudaSuccess)
        per_sm = 1;
    return cfg.search_blocks > 0 ? cfg.search_blocks : g->sm_count * std::max(1, per_sm);
}

// Capture R rounds (commit + search, alternating window buffers from 0) and the control-word
// read into g->round_exec, updating the executable graph in place when only the kernel
// parameters changed.  Returns 0 on success; on any failure the stream is left out of capture,
// the error is cleared, and the caller launches the kernels one by one.
static void launch_commit(const Batch &B, int q, bool small, int commit_blocks, size_t smem, cudaStream_t stream) {
    if (small)
        k_commit<KMAP_SMALL><<<commit_blocks, COMMIT_THREADS_SMALL, smem, stream>>>(B, q);
    else
        k_commit<KMAP><<<commit_blocks, COMMIT_THREADS, smem, stream>>>(B, q);
}

static void launch_search(const Batch &B, int q, int sblocks, cudaStream_t stream) {
    k_search<<<sblocks, SEARCH_THREADS, 0, stream>>>(B, q);
}

static int capture_rounds(DeviceGraph *g, const Batch &B, int R, bool small, int commit_blocks, size_t smem,
                          int sblocks, cudaStream_t stream, Ctl *h_ctl, Ctl *d_ctl,
                          const cudaEvent_t *tev) {
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    for (int r = 0; r < R; r++) {
        launch_commit(B, r & 1, small, commit_blocks, smem, stream);
        // an event record node needs the external flag (a plain record inside a capture only
        // orders streams)
        if (tev) cudaEventRecordWithFlags(tev[2 * r], stream, cudaEventRecordExternal);
        launch_search(B, r & 1, sblocks, stream);
        if (tev) cudaEventRecordWithFlags(tev[2 * r + 1], stream, cudaEventRecordExternal);
    }
    cudaMemcpyAsync(h_ctl, d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream);
    const cudaError_t ce = cudaStreamEndCapture(stream, &gr);
    if (ce != cudaSuccess || gr == nullptr) {
        if (gr) cudaGraphDestroy(gr);
        (void)cudaGetLastError();
        return 1;
    }
    bool ok = false;
    if (g->round_exec) {
        cudaGraphExecUpdateResultInfo info;
        ok = cudaGraphExecUpdate(g->round_exec, gr, &info) == cudaSuccess;
        if (!ok) {
            (void)cudaGetLastError();
            cudaGraphExecDestroy(g->round_exec);
            g->round_exec = nullptr;
        }
    }
    if (!ok) {
        ok = cudaGraphInstantiate(&g->round_exec, gr, 0) == cudaSuccess;
        if (!ok) {
            (void)cudaGetLastError();
            g->round_exec = nullptr;
        }
        g->graph_instantiations += ok;
    }
    cudaGraphDestroy(gr);
    return ok ? 0 : 1;
}

int dev_eval(DeviceGraph *g, const Plan *d_plans, int32_t P, flexis_support_result *d_results,
             cudaStream_t stream, const EvalConfig &cfg, flexis_stats *stats) {
    if (P <= 0) return FLEXIS_OK;
    const auto t_start = std::chrono::steady_clock::now();
    CK(cudaSetDevice(g->device));
    const int Wmax = std::max(32, std::min(cfg.w_max, 16384));
    const int Wmin = std::max(1, std::min(cfg.w_min, Wmax));
    int rc = ws_ensure(g, g->ws, P, Wmax, cfg.record_selected);
    if (rc) return rc;
    Workspace &w = g->ws;
    g->last_P = P;
    g->last_sel = cfg.record_selected;
    Batch B = make_batch(g, w, d_plans, P, Wmin, Wmax, cfg.record_selected, d_results);
    // large batches walk a list of the patterns still active; small ones launch a block per slot
    const int list_threshold = 4 * g->sm_count;
    if (P > list_threshold) B.alist = w.alist;
    // large batches with windows of <= 1024 slots: the small-horizon commit, one full wave
    const bool small_commit = P > list_threshold && Wmax <= SMALL_COMMIT_WMAX;
    const int commit_blocks = small_commit ? g->commit_small_blocks : P > list_threshold ? list_threshold : P;
    if (cfg.search_budget != 0) B.budget = cfg.search_budget < 0 ? 0u : (uint32_t)cfg.search_budget;
    if (cfg.split_pieces != 0) B.split_max = cfg.split_pieces < 0 ? 0 : std::min(cfg.split_pieces, SPLIT_MAX);
    if (cfg.sub_searches > 0) {
        const int k = std::min(cfg.sub_searches, KSUSP);
        B.sid_all = k >= 32 ? 0xFFFFFFFFu : ((1u << k) - 1u);
    }
    const size_t smem = small_commit ? commit_smem_of<KMAP_SMALL>() : commit_smem(Wmax);
    const int sblocks = search_grid(g, cfg);
    B.deadline_ns = cfg.deadline_ms > 0 ? (unsigned long long)cfg.deadline_ms * 1000000ull : 0ull;

    int64_t launches = 0;
    CK(cudaEventRecord(g->ev[0], stream));
    // used bitmaps: only those not known to be zero are cleared here (the previous evaluation
    // cleaned up after itself); until this one cleans up, none is known to be zero
    const int32_t clean0 = w.clean;
    w.clean = 0;
    if (clean0 < P)
        CK(cudaMemsetAsync(w.used + (size_t)g->view.words * clean0, 0,
                           sizeof(uint32_t) * (size_t)g->view.words * (P - clean0), stream));
    CK(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), stream));
    k_init<<<(P + 255) / 256, 256, 0, stream>>>(B);
    launches += 1;
    int64_t rounds = 0;
    int search_launches = 0;
    int R = std::max(1, cfg.rounds_per_sync);
    size_t evi = 0;
    // The R rounds between two host checks (commit + search each, then the control-word read)
    // are captured once per level into a CUDA graph and replayed: the round loop's launches
    // cost one graph launch per R rounds.  R is even so that the window buffer parity of a
    // replay matches the rounds it stands for.
    // With timing, the graph also records an event pair around each search launch; the pairs
    // are read after every replay.
    const bool use_graph = cfg.graphs && stream != nullptr && stream != cudaStreamLegacy &&
                           stream != cudaStreamPerThread;
    bool graph_done = false;
    int64_t graph_launches = 0;
    float graph_search_ms = 0.f;
    // the deadline is checked where the host waits anyway (between groups of rounds)
    bool timed_out = false;
    auto past_deadline = [&]() {
        if (cfg.deadline_ms <= 0) return false;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        timed_out = ms > cfg.deadline_ms;
        return timed_out;
    };
    if (use_graph) {
        R += R & 1;
        while (cfg.timing && g->gev.size() < (size_t)(2 * R)) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            g->gev.push_back(e);
        }
        if (!capture_rounds(g, B, R, small_commit, commit_blocks, smem, sblocks, stream,
                            w.h_ctl, w.ctl,
                            cfg.timing ? g->gev.data() : nullptr)) {
            for (;;) {
                CK(cudaGraphLaunch(g->round_exec, stream));
                launches += 2 * R;
                search_launches += R;
                rounds += R;
                CK(cudaStreamSynchronize(stream));
                graph_launches++;
                if (cfg.timing) {
                    for (int r = 0; r < R; r++) {
                        float x = 0.f;
                        CK(cudaEventElapsedTime(&x, g->gev[2 * r], g->gev[2 * r + 1]));
                        graph_search_ms += x;
                    }
                }
                if (w.h_ctl->active[(rounds - 1) & 1] == 0) break;
                if (past_deadline()) break;
            }
            graph_done = true;
        } else {
            g->graph_fallbacks++;
        }
    }
    if (!graph_done) for (;;) {
        for (int r = 0; r < R; r++) {
            const int q = (int)(rounds & 1);
            launch_commit(B, q, small_commit, commit_blocks, smem, stream);
            if (cfg.timing) {
                while (evi + 2 > g->sev.size()) {
                    cudaEvent_t e;
                    CK(cudaEventCreate(&e));
                    g->sev.push_back(e);
                }
                CK(cudaEventRecord(g->sev[evi], stream));
            }
            launch_search(B, q, sblocks, stream);
            if (cfg.timing) {
                CK(cudaEventRecord(g->sev[evi + 1], stream));
                evi += 2;
            }
            launches += 2;
            search_launches++;
            rounds++;
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        if (w.h_ctl->active[(rounds - 1) & 1] == 0) break;
        if (past_deadline()) break;
    }
    if (timed_out) {
        k_cancel<<<(P + 255) / 256, 256, 0, stream>>>(B, nullptr, P);
        launches += 1;
    }
    cudaEvent_t m0 = nullptr, m1 = nullptr;
    if (cfg.timing) {
        CK(cudaEventCreate(&m0));
        CK(cudaEventCreate(&m1));
    }
    k_mni_setup<<<1, 1024, 0, stream>>>(B);
    if (cfg.timing) CK(cudaEventRecord(m0, stream));
    k_mni<<<sblocks, SEARCH_THREADS, 0, stream>>>(B);
    if (cfg.timing) CK(cudaEventRecord(m1, stream));
    k_finalize<<<(P + 255) / 256, 256, 0, stream>>>(B);
    k_clear_used<<<(int)(((int64_t)P * 32 + 255) / 256), 256, 0, stream>>>(B);
    launches += 4;
    CK(cudaGetLastError());
    w.clean = std::max(clean0, P);
    flexis_stats est{};
    if (cfg.count_maps || cfg.exact_mis) {
        const int rc2 = dev_enumerate(g, d_plans, P, d_results, stream, cfg, &est, t_start);
        if (rc2) return rc2;
    }
    CK(cudaEventRecord(g->ev[1], stream));
    CK(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->rounds = rounds;
        stats->search_items = (int64_t)w.h_ctl->search_items;
        stats->mni_items = (int64_t)w.h_ctl->mni_items;
        stats->kernel_launches = launches;
        stats->alg_bytes_greedy = (int64_t)w.h_ctl->bytes_greedy;
        stats->alg_bytes = (int64_t)(w.h_ctl->bytes_greedy + w.h_ctl->bytes_mni);
        stats->search_scanned = (int64_t)w.h_ctl->alg_scanned;
        stats->search_bound = (int64_t)w.h_ctl->alg_bound;
        stats->search_map_words = (int64_t)w.h_ctl->alg_map_words;
        stats->search_launches = search_launches;
        stats->graph_launches = (int32_t)graph_launches;
        stats->d2h_bytes = (int64_t)sizeof(Ctl) * (rounds / R + 1);  // control-word reads
        stats->kernel_launches += est.kernel_launches;
        stats->enum_rows = est.enum_rows;
        stats->enum_scanned = est.enum_scanned;
        stats->enum_bytes = est.enum_bytes;
        float t = 0.f;
        cudaEventElapsedTime(&t, g->ev[0], g->ev[1]);
        stats->total_ms = t;
        if (cfg.timing) {
            float sum = 0.f;
            for (size_t k = 0; k < evi; k += 2) {
                float x = 0.f;
                cudaEventElapsedTime(&x, g->sev[k], g->sev[k + 1]);
                sum += x;
            }
            stats->search_ms = sum + graph_search_ms;
            float y = 0.f;
            cudaEventElapsedTime(&y, m0, m1);
            stats->mni_ms = y;
        }
    }
    if (m0) cudaEventDestroy(m0);
    if (m1) cudaEventDestroy(m1);
    return FLEXIS_OK;
}

int dev_eval_host(DeviceGraph *g, const Plan *h_plans, int32_t P, flexis_support_result *h_results,
                  const EvalConfig &cfg, flexis_stats *stats) {
    if (P <= 0) return FLEXIS_OK;
    CK(cudaSetDevice(g->device));
    Workspace &w = g->ws;
    int rc = ws_ensure(g, w, P, std::max(32, std::min(cfg.w_max, 16384)), cfg.record_selected);
    if (rc) return rc;
    CK(cudaMemcpyAsync(w.plans, h_plans, sizeof(Plan) * (size_t)P, cudaMemcpyHostToDevice, g->stream));
    rc = dev_eval(g, w.plans, P, w.results, g->stream, cfg, stats);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h_results, w.results, sizeof(flexis_support_result) * (size_t)P,
                       cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (stats) {
        stats->h2d_bytes += (int64_t)sizeof(Plan) * P;
        stats->d2h_bytes += (int64_t)sizeof(flexis_support_result) * P;
    }
    return FLEXIS_OK;
}

// ------------------------------------------------------------------ allocation-free evaluation
// One pattern evaluated with all of its device scratch (control words, pattern state, plan,
// result, window buffers, work items, saved searches, used-vertex bitmap) carved out of a single
// statically allocated device array, so the call itself allocates nothing.  The array belongs to
// the module: every GPU that loads the library holds it until the process exits, and every call
// on a device reuses the same bytes.
constexpr size_t NOALLOC_SCRATCH_BYTES = 8ull << 20;  // 8 MiB per device
constexpr int NOALLOC_WMAX = 1024;                    // speculation window of this entry point
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

struct NoallocLayout {
    size_t ctl, st, plan, result, mni_seg, items, win_root, win_state, win_map, susp, used, end;
};

static NoallocLayout noalloc_layout(int64_t words) {
    NoallocLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    L.ctl = take(sizeof(Ctl));
    L.st = take(sizeof(PatState));
    L.plan = take(sizeof(Plan));
    L.result = take(sizeof(flexis_support_result));
    L.mni_seg = take(sizeof(unsigned long long) * (MAXN + 1));
    L.items = take(sizeof(int2) * (NOALLOC_WMAX + KSUSP));
    L.win_root = take(sizeof(int32_t) * 2 * NOALLOC_WMAX);
    L.win_state = take(sizeof(int32_t) * 2 * NOALLOC_WMAX);
    L.win_map = take(sizeof(int32_t) * 2 * NOALLOC_WMAX * MAXN);
    L.susp = take(sizeof(uint32_t) * KSUSP * DFS_SAVE_STRIDE);
    L.used = take(sizeof(uint32_t) * (size_t)words);
    L.end = off;
    return L;
}

int64_t noalloc_max_vertices() {
    const NoallocLayout L = noalloc_layout(0);
    return (int64_t)(NOALLOC_SCRATCH_BYTES - L.used) / 4 * 32;
}

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_base[256];  // device address of the scratch array, per device

// Set-up, once per device and with that device current: the device address of the array.  In
// host code the array's name is only a host-side stand-in, so kernels get this address instead.
static int noalloc_base(int device, unsigned char **out) {
    if (device < 0 || device >= 256) return FLEXIS_E_INVALID;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "flexis: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return FLEXIS_E_CUDA;
        }
        g_noalloc_base[device] = (unsigned char *)p;
    }
    *out = g_noalloc_base[device];
    return FLEXIS_OK;
}

int dev_support_noalloc(DeviceGraph *g, const Plan *h_plan, flexis_support_result *h_out,
                        cudaStream_t stream, int32_t deadline_ms) {
    const auto t_start = std::chrono::steady_clock::now();
    CK(cudaSetDevice(g->device));
    const NoallocLayout L = noalloc_layout(g->view.words);
    if (L.end > NOALLOC_SCRATCH_BYTES) {
        fprintf(stderr, "flexis: flexis_support_noalloc supports graphs of at most %lld vertices "
                        "(this graph has %lld)\n", (long long)noalloc_max_vertices(), (long long)g->view.nv);
        return FLEXIS_E_UNSUPPORTED;
    }
    unsigned char *base = nullptr;
    int rc = noalloc_base(g->device, &base);
    if (rc) return rc;
    if (!stream) stream = g->stream;
    Batch B{};  // every field zero (null pointers: no active list, no selection log) unless set below
    B.G = g->view;
    B.plans = reinterpret_cast<const Plan *>(base + L.plan);
    B.P = 1;
    B.Wmax = NOALLOC_WMAX;
    B.Wmin = 256;
    B.sel_cap = 0;
    B.budget = SEARCH_BUDGET;
    B.split_max = SPLIT_MAX;
    B.sid_all = KSUSP >= 32 ? 0xFFFFFFFFu : ((1u << (KSUSP & 31)) - 1u);
    B.st = reinterpret_cast<PatState *>(base + L.st);
    B.used = reinterpret_cast<uint32_t *>(base + L.used);
    B.win_root = reinterpret_cast<int32_t *>(base + L.win_root);
    B.win_state = reinterpret_cast<int32_t *>(base + L.win_state);
    B.win_map = reinterpret_cast<int32_t *>(base + L.win_map);
    B.items = reinterpret_cast<int2 *>(base + L.items);
    B.ctl = reinterpret_cast<Ctl *>(base + L.ctl);
    B.sel = nullptr;
    B.mni_seg = reinterpret_cast<unsigned long long *>(base + L.mni_seg);
    B.susp = reinterpret_cast<uint32_t *>(base + L.susp);
    B.results = reinterpret_cast<flexis_support_result *>(base + L.result);
    B.deadline_ns = deadline_ms > 0 ? (unsigned long long)deadline_ms * 1000000ull : 0ull;
    // the scratch keeps the previous call's contents: the used bitmap must start empty (the
    // pattern state and control words are rewritten by k_init)
    CK(cudaMemcpyAsync(base + L.plan, h_plan, sizeof(Plan), cudaMemcpyHostToDevice, stream));
    CK(cudaMemsetAsync(B.used, 0, sizeof(uint32_t) * (size_t)g->view.words, stream));
    CK(cudaMemsetAsync(B.ctl, 0, sizeof(Ctl), stream));
    k_init<<<1, 256, 0, stream>>>(B);
    const int sblocks = g->sm_count * 6;
    Ctl h_ctl;
    for (int64_t round = 0;;) {
        for (int r = 0; r < 2; r++, round++) {
            const int q = (int)(round & 1);
            k_commit<KMAP><<<1, COMMIT_THREADS, commit_smem(0), stream>>>(B, q);
            k_search<<<sblocks, SEARCH_THREADS, 0, stream>>>(B, q);
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&h_ctl, B.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        if (h_ctl.active[(round - 1) & 1] == 0) break;
        // the graph's deadline, checked between pairs of rounds as in dev_eval: an undecided
        // pattern stops with FLEXIS_E_TIMEOUT
        if (deadline_ms > 0 &&
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count() > deadline_ms) {
            k_cancel<<<1, 32, 0, stream>>>(B, nullptr, 1);
            break;
        }
    }
    k_mni_setup<<<1, 1024, 0, stream>>>(B);
    k_mni<<<sblocks, SEARCH_THREADS, 0, stream>>>(B);
    k_finalize<<<1, 256, 0, stream>>>(B);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h_out, B.results, sizeof(flexis_support_result), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return FLEXIS_OK;
}

int dev_selected(DeviceGraph *g, int32_t i, int32_t *maps_out, int64_t cap, int64_t *n_out) {
    if (i < 0 || i >= g->last_P || g->last_sel <= 0 || !g->ws.sel_buf) return FLEXIS_E_INVALID;
    CK(cudaSetDevice(g->device));
    PatState s;
    CK(cudaMemcpy(&s, g->ws.st + i, sizeof s, cudaMemcpyDeviceToHost));
    int64_t n = std::min<int64_t>(s.logged, cap);
    if (n > 0)
        CK(cudaMemcpy(maps_out, g->ws.sel_buf + (size_t)i * g->last_sel * MAXN,
                      sizeof(int32_t) * n * MAXN, cudaMemcpyDeviceToHost));
    *n_out = n;
    return FLEXIS_OK;
}

// ------------------------------------------------------------------ serving session
// Continuous batching at round granularity: each step admits new plans into free slots, runs
// one speculation round over every slot still in its greedy phase, runs the MNI search for the
// slots that finished their greedy phase in that round, and returns every slot's phase and
// result.  Requests admitted at different steps share the device rounds.
constexpr int SERVE_WMAX = 2048;
constexpr int SERVE_BUDGET = 256;

struct ServeSession {
    DeviceGraph *g = nullptr;
    Workspace w;
    cudaStream_t stream = nullptr;
    int32_t slots = 0;
    // A request starts at a window of Wmin roots, doubling up to Wmax while its speculation
    // stays conflict-free.  Rounds are shared by every request in flight, so a round lasts as
    // long as its longest search: the per-round search budget is much smaller than a batch's
    // (measured on the MiCo-shaped serving stream: 4096 -> 256 chunks cut p50 from 49 to 8 ms
    // and p99 from 435 to 161 ms, and raised the saturated throughput 1.7x).
    int Wmin = 32, Wmax = SERVE_WMAX;
    int32_t budget = SERVE_BUDGET;
    int32_t *d_admit = nullptr;
    int32_t *h_admit = nullptr;  // pinned
    int32_t *d_cancel = nullptr;
    int32_t *h_cancel = nullptr;  // pinned
    Plan *h_plans = nullptr;     // pinned staging
    PatState *h_st = nullptr;    // pinned
    flexis_support_result *h_res = nullptr;  // pinned
    int64_t round = 0;
    int sblocks = 0;
};

int serve_create(DeviceGraph *g, int32_t slots, int32_t wmin, int32_t wmax, int32_t budget,
                 ServeSession **out) {
    CK(cudaSetDevice(g->device));
    ServeSession *s = new ServeSession();
    s->g = g;
    s->slots = slots;
    if (wmax > 0) s->Wmax = std::max(32, std::min(wmax, 16384));
    if (wmin > 0) s->Wmin = std::max(1, std::min(wmin, s->Wmax));
    if (budget != 0) s->budget = budget;
    int rc = ws_ensure(g, s->w, slots, s->Wmax, 0);
    if (rc) { serve_destroy(s); return rc; }
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&s->d_admit, sizeof(int32_t) * slots) != cudaSuccess ||
        cudaMallocHost((void **)&s->h_admit, sizeof(int32_t) * slots) != cudaSuccess ||
        cudaMalloc(&s->d_cancel, sizeof(int32_t) * slots) != cudaSuccess ||
        cudaMallocHost((void **)&s->h_cancel, sizeof(int32_t) * slots) != cudaSuccess ||
        cudaMallocHost((void **)&s->h_plans, sizeof(Plan) * slots) != cudaSuccess ||
        cudaMallocHost((void **)&s->h_st, sizeof(PatState) * slots) != cudaSuccess ||
        cudaMallocHost((void **)&s->h_res, sizeof(flexis_support_result) * slots) != cudaSuccess) {
        serve_destroy(s);
        return FLEXIS_E_NOMEM;
    }
    memset(s->h_st, 0, sizeof(PatState) * slots);  // host view: every slot free
    EvalConfig cfg;
    s->sblocks = search_grid(g, cfg);
    // every slot starts free
    CK(cudaMemsetAsync(s->w.st, 0, sizeof(PatState) * slots, s->stream));
    Batch B = make_batch(g, s->w, s->w.plans, slots, s->Wmin, s->Wmax, 0, s->w.results);
    k_reset_ctl<<<1, 1, 0, s->stream>>>(B);
    CK(cudaStreamSynchronize(s->stream));
    *out = s;
    return FLEXIS_OK;
}

void serve_destroy(ServeSession *s) {
    if (!s) return;
    cudaSetDevice(s->g->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    ws_free(s->w);
    cudaFree(s->d_admit);
    if (s->h_admit) cudaFreeHost(s->h_admit);
    cudaFree(s->d_cancel);
    if (s->h_cancel) cudaFreeHost(s->h_cancel);
    if (s->h_plans) cudaFreeHost(s->h_plans);
    if (s->h_st) cudaFreeHost(s->h_st);
    if (s->h_res) cudaFreeHost(s->h_res);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int serve_slot_bytes(const DeviceGraph *g, int32_t wmax, int64_t *bytes) {
    const int64_t W = wmax > 0 ? std::max(32, std::min(wmax, 16384)) : ServeSession().Wmax;
    *bytes = (int64_t)g->view.words * 4 + W * (2 * (4 + 4 + 4 * MAXN) + 8) + (int64_t)sizeof(PatState) +
             (int64_t)sizeof(Plan);
    return FLEXIS_OK;
}

// Stop the listed requests before the next step (their deadline passed); that step finalises
// them with FLEXIS_E_TIMEOUT.
int serve_cancel(ServeSession *s, const int32_t *slots, int32_t n) {
    if (n <= 0) return FLEXIS_OK;
    DeviceGraph *g = s->g;
    CK(cudaSetDevice(g->device));
    memcpy(s->h_cancel, slots, sizeof(int32_t) * (size_t)n);
    CK(cudaMemcpyAsync(s->d_cancel, s->h_cancel, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s->stream));
    Batch B = make_batch(g, s->w, s->w.plans, s->slots, s->Wmin, s->Wmax, 0, s->w.results);
    k_cancel<<<(n + 255) / 256, 256, 0, s->stream>>>(B, s->d_cancel, n);
    CK(cudaGetLastError());
    return FLEXIS_OK;
}

int serve_step(ServeSession *s, const int32_t *admit_slots, const Plan *admit_plans, int32_t n_admit,
               int32_t *phase_out, flexis_support_result *res_out, int32_t *n_greedy) {
    DeviceGraph *g = s->g;
    CK(cudaSetDevice(g->device));
    Batch B = make_batch(g, s->w, s->w.plans, s->slots, s->Wmin, s->Wmax, 0, s->w.results);
    B.budget = s->budget < 0 ? 0u : (uint32_t)s->budget;
    for (int32_t i = 0; i < n_admit; i++) {
        s->h_admit[i] = admit_slots[i];
        s->h_plans[i] = admit_plans[i];
        CK(cudaMemcpyAsync(s->w.plans + admit_slots[i], &s->h_plans[i], sizeof(Plan),
                           cudaMemcpyHostToDevice, s->stream));
    }
    if (n_admit > 0) {
        CK(cudaMemcpyAsync(s->d_admit, s->h_admit, sizeof(int32_t) * n_admit, cudaMemcpyHostToDevice, s->stream));
        k_admit<<<n_admit, 256, 0, s->stream>>>(B, s->d_admit, n_admit);
    }
    const int q = (int)(s->round & 1);
    k_commit<KMAP><<<s->slots, COMMIT_THREADS, commit_smem(s->Wmax), s->stream>>>(B, q);
    k_search<<<s->sblocks, SEARCH_THREADS, 0, s->stream>>>(B, q);
    s->round++;
    k_mni_setup<<<1, 1024, 0, s->stream>>>(B);
    k_mni<<<s->sblocks, SEARCH_THREADS, 0, s->stream>>>(B);
    k_finalize<<<(s->slots + 255) / 256, 256, 0, s->stream>>>(B);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(s->h_st, s->w.st, sizeof(PatState) * s->slots, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(s->h_res, s->w.results, sizeof(flexis_support_result) * s->slots,
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    int32_t ng = 0;
    for (int32_t i = 0; i < s->slots; i++) {
        phase_out[i] = s->h_st[i].phase;
        if (s->h_st[i].phase == PH_GREEDY) ng++;
        if (s->h_st[i].phase == PH_READY) res_out[i] = s->h_res[i];
    }
    *n_greedy = ng;
    return FLEXIS_OK;
}

}  // namespace fx
