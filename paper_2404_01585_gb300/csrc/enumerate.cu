// Level-by-level enumeration of every map of a batch of patterns (the set M of Sec. 2.4), for
// the map count n_maps (FLEXIS_MODE_COUNT_MAPS) and for materialising the maps whose overlap
// graph the exact maximum-independent-set search works on (FLEXIS_MODE_EXACT_MIS).
//
// Unlike the greedy search of kernels.cu, which stops at the first map of each root, this path
// keeps every partial map: level i of the frontier holds rows [pattern, t_0 .. t_i] (the data
// vertices bound to the first i+1 levels of the pattern's matching order).  One warp extends one
// row: it finds the label slices of the row's bound neighbours of level i+1, scans the shortest
// one 32 candidates at a time (coalesced loads), tests each candidate against the others by
// binary search, against injectivity and against the one-hop label/degree filter, and keeps the
// survivors (ballot).  The survivors of a chunk are staged in shared memory and written out as
// one contiguous, coalesced block of rows.
//
// The frontier of a level is capped (options.frontier_rows, at least the largest degree): a
// count pass gives each row's survivor count, an exclusive scan gives output offsets, and the
// write pass extends a prefix of rows whose survivors fit, after which the next level is
// processed before the rest of the current one (depth-first over capped breadth-first chunks).
// Rows of the last level are never written: their survivors are counted (and, for exact-MIS
// patterns, copied to a per-pattern map buffer).  Every row's output lands at its scan offset,
// so the frontier is in lexicographic order and the result does not depend on scheduling.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>

#include "fx_kern.cuh"

namespace fx {

constexpr int ENUM_THREADS = 256;
constexpr int ENUM_WARPS = ENUM_THREADS / 32;
constexpr int64_t ENUM_DEFAULT_ROWS = 1ll << 22;
constexpr unsigned long long DEFAULT_MAPS_CAP = 1ull << 32;

// Algorithmic counters of the enumerator (device): rows extended, driver-slice entries scanned,
// survivors, and bytes read (slices, records, probes).
enum { EST_ROWS = 0, EST_SCANNED = 1, EST_SURVIVORS = 2, EST_BYTES = 3, EST_N = 4 };

struct EnumPass {
    DevGraphView G;
    const Plan *plans;
    int32_t P;
    int32_t level;                          // input rows hold levels 0..level
    const int32_t *in;                      // level >= 1: rows of level + 2 ints
    const unsigned long long *root_prefix;  // level 0: [P + 1] prefix of the patterns' root counts
    long long row0, nrows;                  // input rows [row0, row0 + nrows)
    unsigned long long *cnt;                // count pass: survivors of each non-final row
    const unsigned long long *off;          // write pass: exclusive prefix of cnt (nrows + 1)
    int32_t *out;                           // write pass: rows of level + 3 ints
    unsigned long long *n_maps;             // [P] maps counted
    unsigned long long maps_cap;
    int32_t *maps;                          // [P][maps_per][MAXN] materialised maps (nullable)
    unsigned long long *maps_n;             // [P] maps materialised (may pass maps_per: overflow)
    int32_t maps_per;
    unsigned long long *next;               // row counter of this launch
    unsigned long long *stat;               // [EST_N]
};

__device__ __forceinline__ bool enum_wanted(const Plan &P) {
    return P.status == FLEXIS_OK && !(P.flags & FLEXIS_FLAG_ABSENT_LABEL) && (P.count_maps || P.exact_mis);
}

// A pattern stops being enumerated once its count saturated and (for exact MIS) its map buffer
// overflowed: nothing further can change its results.
__device__ __forceinline__ bool enum_stopped(const EnumPass &E, const Plan &P, int p) {
    const bool count_done = !P.count_maps || __ldcg(E.n_maps + p) >= E.maps_cap;
    const bool maps_done = !P.exact_mis || !E.maps || __ldcg(E.maps_n + p) > (unsigned long long)E.maps_per;
    return count_done && maps_done;
}

// Root counts of the enumerated patterns and their prefix (virtual level-0 rows).
__global__ void k_enum_prefix(const Plan *plans, int32_t P, unsigned long long *prefix) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < P; base += blockDim.x) {
        const int p = base + tid;
        unsigned long long v = 0;
        if (p < P && enum_wanted(plans[p])) v = (unsigned long long)max(0, plans[p].root_end - plans[p].root_begin);
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULLMASK, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned long long t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULLMASK, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const unsigned long long excl = carry + x - v + (w > 0 ? warp_tot[w - 1] : 0);
        if (p < P) prefix[p] = excl;
        __syncthreads();
        if (tid == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (tid == 0) prefix[P] = carry;
}

// Extend rows of level E.level by one level.  WRITE = false: count pass (per-row survivor counts
// of non-final rows; last-level survivors counted into n_maps and materialised for exact MIS).
// WRITE = true: write pass (survivors of non-final rows written at their scan offsets).
template <bool WRITE>
__global__ void __launch_bounds__(ENUM_THREADS) k_extend(EnumPass E) {
    __shared__ WarpState ws[ENUM_WARPS];
    __shared__ int32_t stage[ENUM_WARPS][32 * (MAXN + 1)];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpState &W = ws[wid];
    int32_t *sg = stage[wid];
    const int i = E.level, j = i + 1;
    const int in_w = i + 2, out_w = i + 3;  // row widths (pattern id + vertices)
    unsigned long long bytes = 0, scanned = 0, surv = 0, rows = 0;
    uint32_t probes = 0;
    for (;;) {
        unsigned long long r = 0;
        if (lane == 0) r = atomicAdd(E.next, 1ull);
        r = __shfl_sync(FULLMASK, r, 0);
        if (r >= (unsigned long long)E.nrows) break;
        if (WRITE && E.off[r + 1] == E.off[r]) continue;  // final row or no survivor
        const long long row = E.row0 + (long long)r;
        int p;
        int32_t x = 0;
        if (i == 0) {
            // virtual row: the (row - prefix[p])-th root of pattern p
            int lo = 0, hi = E.P;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (E.root_prefix[mid] <= (unsigned long long)row) lo = mid; else hi = mid;
            }
            p = lo;
            if (lane == 1) x = __ldg(E.G.lab_vtx + E.plans[p].root_begin + (row - (long long)E.root_prefix[p]));
        } else {
            const int32_t *src = E.in + row * in_w;
            x = lane < in_w ? src[lane] : 0;
            p = __shfl_sync(FULLMASK, x, 0);
        }
        const Plan &P = E.plans[p];
        // the count pass drops rows of patterns that need nothing more; the write pass never
        // does (the row's output slots are reserved and must hold valid rows)
        if (!WRITE && enum_stopped(E, P, p)) {
            if (lane == 0) E.cnt[r] = 0;
            continue;
        }
        load_level_plan(W, P.greedy, P);
        if (lane >= 1 && lane <= j) W.t[lane - 1] = x;
        __syncwarp();
        rows++;
        const bool final = j == P.n - 1;
        bool ok = true;
        if (i == 0) {
            bytes += 32;
            ok = vertex_fits(E.G, W.t[0], W.L.deg[0], W.need[W.L.vert[0]]);
        }
        if (ok) ok = enter_level(E.G, W, j, bytes);
        unsigned long long total = 0;
        unsigned long long wbase = WRITE ? E.off[r] - E.off[0] : 0;
        if (ok) {
            const uint32_t lo = W.lo[j], hi = W.hi[j];
            for (uint32_t pos = lo; pos < hi; pos += 32) {
                const uint32_t k = pos + lane;
                int32_t c = -1;
                bool good = false;
                uint32_t rej = 0;
                if (k < hi) {
                    c = __ldg(E.G.adj + k);
                    good = check_candidate(E.G, W, j, c, nullptr, probes, rej);
                }
                const unsigned mask = __ballot_sync(FULLMASK, good);
                scanned += min(32u, hi - pos);
                if (!mask) continue;
                const int nm = __popc(mask);
                const int q = __popc(mask & ((1u << lane) - 1u));  // rank of this survivor
                total += nm;
                if (!WRITE && final && P.exact_mis && E.maps) {
                    unsigned long long b0 = 0;
                    if (lane == 0) b0 = atomicAdd(E.maps_n + p, (unsigned long long)nm);
                    b0 = __shfl_sync(FULLMASK, b0, 0);
                    const unsigned long long idx = b0 + q;
                    if (good && idx < (unsigned long long)E.maps_per) {
                        int32_t *m = E.maps + ((size_t)p * E.maps_per + idx) * MAXN;
                        for (int l = 0; l < MAXN; l++) m[l] = l < j ? W.t[l] : (l == j ? c : -1);
                    }
                }
                if (WRITE && !final) {
                    // stage the chunk's rows in shared memory, then write them as one block
                    if (good) {
                        int32_t *o = sg + q * out_w;
                        o[0] = p;
                        for (int l = 0; l < j; l++) o[1 + l] = W.t[l];
                        o[1 + j] = c;
                    }
                    __syncwarp();
                    int32_t *dst = E.out + (size_t)wbase * out_w;
                    for (int w = lane; w < nm * out_w; w += 32) dst[w] = sg[w];
                    wbase += nm;
                    __syncwarp();
                }
            }
        }
        surv += total;
        if (!WRITE && lane == 0) {
            if (final) {
                E.cnt[r] = 0;
                if (total) atomicAdd(E.n_maps + p, total);
            } else {
                E.cnt[r] = total;
            }
        }
    }
    const unsigned long long pb = warp_sum((unsigned long long)probes * 4ull);
    if (lane == 0 && !WRITE) {
        atomicAdd(E.stat + EST_ROWS, rows);
        atomicAdd(E.stat + EST_SCANNED, scanned);
        atomicAdd(E.stat + EST_SURVIVORS, surv);
        atomicAdd(E.stat + EST_BYTES, bytes + pb + 4ull * scanned);
    }
}

// Exclusive scan of cnt[0, n) into off[0, n] (off[n] = total), three launches.
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long &total,
                                                            unsigned long long *sh /* >= 33 */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULLMASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULLMASK, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sh[lane] = t;
        if (lane == nw - 1) sh[32] = t;
    }
    __syncthreads();
    const unsigned long long excl = x - v + (w > 0 ? sh[w - 1] : 0);
    total = sh[32];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const unsigned long long *cnt, unsigned long long *off,
                                                     long long n, unsigned long long *tsum) {
    __shared__ unsigned long long sh[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    const long long a = base + 2 * threadIdx.x;
    const unsigned long long v0 = a < n ? cnt[a] : 0, v1 = a + 1 < n ? cnt[a + 1] : 0;
    unsigned long long tot;
    const unsigned long long ex = block_scan_u64(v0 + v1, tot, sh);
    if (a < n) off[a] = ex;
    if (a + 1 < n) off[a + 1] = ex + v0;
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_tops(unsigned long long *tsum, int ntiles, unsigned long long *off,
                                                    long long n) {
    __shared__ unsigned long long sh[33];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < ntiles; b += blockDim.x) {
        const int t = b + threadIdx.x;
        const unsigned long long v = t < ntiles ? tsum[t] : 0;
        unsigned long long tot;
        const unsigned long long ex = block_scan_u64(v, tot, sh);
        if (t < ntiles) tsum[t] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void k_scan_add(unsigned long long *off, long long n, const unsigned long long *tsum) {
    const long long a = (long long)blockIdx.x * SCAN_TILE + threadIdx.x;
    const unsigned long long add = tsum[blockIdx.x];
    for (long long x = a; x < min(n, (long long)(blockIdx.x + 1) * SCAN_TILE); x += blockDim.x) off[x] += add;
}

int dev_scan_u64(unsigned long long *cnt_off, long long n, unsigned long long *tsum, cudaStream_t s) {
    const int tiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    if (tiles > 0) k_scan_tiles<<<tiles, 1024, 0, s>>>(cnt_off, cnt_off, n, tsum);
    k_scan_tops<<<1, 1024, 0, s>>>(tsum, tiles, cnt_off, n);
    if (tiles > 0) k_scan_add<<<tiles, 1024, 0, s>>>(cnt_off, n, tsum);
    CK(cudaGetLastError());
    return FLEXIS_OK;
}

// Largest e in (pos, end] with off[e] - off[pos] <= cap (at least pos + 1: one row's survivors
// never exceed the cap, which is at least the largest degree).
__global__ void k_split(const unsigned long long *off, long long pos, long long end, unsigned long long cap,
                        unsigned long long *out) {
    long long lo = pos + 1, hi = end;
    const unsigned long long base = off[pos];
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (off[mid] - base <= cap) lo = mid; else hi = mid - 1;
    }
    *out = (unsigned long long)lo;
}

__global__ void k_enum_finalize(const Plan *plans, int32_t P, flexis_support_result *res,
                                const unsigned long long *n_maps, unsigned long long maps_cap, int timed_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const Plan &Q = plans[p];
    flexis_support_result &r = res[p];
    if (Q.status == FLEXIS_OK && Q.exact_mis && timed_out) {
        // the deadline passed before the maps were complete: a lower bound only
        r.mis_exact = r.mis > 0 ? r.mis : 0;
        r.flags |= FLEXIS_FLAG_EXACT_MIS_SATURATED;
    }
    if (Q.status != FLEXIS_OK || !Q.count_maps) return;
    if (Q.flags & FLEXIS_FLAG_ABSENT_LABEL) {
        r.n_maps = 0;
        return;
    }
    const unsigned long long n = n_maps[p];
    r.n_maps = n < maps_cap ? n : maps_cap;
    if (n >= maps_cap) {
        r.flags |= FLEXIS_FLAG_MAPS_SATURATED;
    } else if (timed_out) {
        r.status = FLEXIS_E_TIMEOUT;
        r.frequent = 0;
    }
}

// ------------------------------------------------------------------ overlap graph and exact MIS
// The maps of an exact-MIS pattern (materialised by the count pass) become its overlap graph
// (Sec. 2.4.1): maps with the same image vertex set (an instance) conflict with each other and
// with the same other maps, so the maximum independent set (Sec. 2.4.2) is taken over distinct
// instances.  One block per pattern:
//   1. each map's image is sorted ascending (one thread per map);
//   2. the maps are sorted lexicographically (bitonic sort of an index array) and deduplicated:
//      the instances, in ascending order;
//   3. the inverted index: keys (vertex << 16 | instance) sorted (bitonic), so the instances
//      holding a data vertex form one run (a segment of equal vertex);
//   4. conflict edges: every pair inside a run sets its bit in the adjacency bitsets.
// Then one warp per pattern runs the branch-and-bound search.
struct ExactArgs {
    const Plan *plans;
    int32_t P;
    int32_t *maps;                     // [P][maps_per][MAXN]
    const unsigned long long *maps_n;  // [P]
    int32_t maps_per;
    int32_t inst_cap;                  // largest instance count searched
    int32_t wcap;                      // words of one adjacency row: (inst_cap + 31) / 32
    int32_t sidx_stride;               // power of two >= maps_per (the sort pads to one)
    int32_t keys_stride;               // power of two >= inst_cap * MAXN
    int32_t *sidx;                     // [P][sidx_stride] sort index
    int32_t *inst;                     // [P][inst_cap][MAXN] instances (sorted rows)
    int32_t *n_inst;                   // [P] instances, -1 when beyond a limit
    unsigned long long *keys;          // [P][keys_stride] inverted-index keys
    uint32_t *adj;                     // [P][inst_cap][wcap] conflict bitsets
    uint32_t *frames;                  // [P][inst_cap + 1][wcap] candidate sets of the search
    int32_t *fmeta;                    // [P][inst_cap + 1][3] size, branch vertex, state
    long long node_budget;
    flexis_support_result *results;
};

__device__ __forceinline__ int row_cmp(const int32_t *a, const int32_t *b) {
    for (int l = 0; l < MAXN; l++)
        if (a[l] != b[l]) return a[l] < b[l] ? -1 : 1;
    return 0;
}

__device__ __forceinline__ unsigned next_pow2(unsigned x) {
    unsigned p = 1;
    while (p < x) p <<= 1;
    return p;
}

__global__ void __launch_bounds__(1024) k_exact_prepare(ExactArgs A) {
    __shared__ int s_n;
    __shared__ int sh_scan[40];
    const int p = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const Plan &Q = A.plans[p];
    if (Q.status != FLEXIS_OK || !Q.exact_mis) return;
    if (Q.flags & FLEXIS_FLAG_ABSENT_LABEL) {
        if (tid == 0) A.n_inst[p] = 0;
        return;
    }
    const unsigned long long mc = A.maps_n[p];
    if (mc > (unsigned long long)A.maps_per) {
        if (tid == 0) A.n_inst[p] = -1;
        return;
    }
    const int n = Q.n, M = (int)mc;
    int32_t *maps = A.maps + (size_t)p * A.maps_per * MAXN;
    int32_t *idx = A.sidx + (size_t)p * A.sidx_stride;
    // 1. sort each image
    for (int t = tid; t < M; t += nt) {
        int32_t *r = maps + (size_t)t * MAXN;
        for (int a = 1; a < n; a++)
            for (int b = a; b > 0 && r[b - 1] > r[b]; b--) {
                const int32_t x = r[b];
                r[b] = r[b - 1];
                r[b - 1] = x;
            }
    }
    // 2. bitonic sort of the map indices by row (padding index -1 sorts last)
    const unsigned M2 = next_pow2((unsigned)max(M, 1));
    for (unsigned t = tid; t < M2; t += nt) idx[t] = t < (unsigned)M ? (int)t : -1;
    __syncthreads();
    auto less_idx = [&](int x, int y) -> bool {  // row(x) < row(y), -1 = +infinity
        if (y < 0) return x >= 0;
        if (x < 0) return false;
        return row_cmp(maps + (size_t)x * MAXN, maps + (size_t)y * MAXN) < 0;
    };
    for (unsigned k = 2; k <= M2; k <<= 1)
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned t = tid; t < M2; t += nt) {
                const unsigned u = t ^ j;
                if (u > t) {
                    const int x = idx[t], y = idx[u];
                    const bool up = (t & k) == 0;
                    if (up ? less_idx(y, x) : less_idx(x, y)) {
                        idx[t] = y;
                        idx[u] = x;
                    }
                }
            }
            __syncthreads();
        }
    // unique rows -> instances (block scan over the first-of-run flags)
    if (tid == 0) s_n = 0;
    __syncthreads();
    int32_t *inst = A.inst + (size_t)p * A.inst_cap * MAXN;
    for (int b0 = 0; b0 < M; b0 += nt) {
        const int t = b0 + tid;
        int first = 0;
        if (t < M) first = (t == 0 || row_cmp(maps + (size_t)idx[t] * MAXN, maps + (size_t)idx[t - 1] * MAXN) != 0);
        int excl;
        const int tot = block_scan(first, excl, sh_scan);
        const int at = s_n + excl;
        if (first && at < A.inst_cap)
            for (int l = 0; l < MAXN; l++) inst[(size_t)at * MAXN + l] = maps[(size_t)idx[t] * MAXN + l];
        __syncthreads();
        if (tid == 0) s_n += tot;
        __syncthreads();
    }
    const int N = s_n;
    if (N > A.inst_cap) {
        if (tid == 0) A.n_inst[p] = -1;
        return;
    }
    // 3. inverted index: (vertex, instance) keys sorted by vertex
    const int K = N * n;
    const unsigned K2 = next_pow2((unsigned)max(K, 1));
    unsigned long long *keys = A.keys + (size_t)p * A.keys_stride;
    for (unsigned t = tid; t < K2; t += nt)
        keys[t] = t < (unsigned)K ? ((unsigned long long)(uint32_t)inst[(size_t)(t / n) * MAXN + t % n] << 16) | (t / n)
                                  : ~0ull;
    // 4a. clear the adjacency rows
    uint32_t *adj = A.adj + (size_t)p * A.inst_cap * A.wcap;
    for (int t = tid; t < N * A.wcap; t += nt) adj[t] = 0u;
    __syncthreads();
    for (unsigned k = 2; k <= K2; k <<= 1)
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned t = tid; t < K2; t += nt) {
                const unsigned u = t ^ j;
                if (u > t) {
                    const unsigned long long x = keys[t], y = keys[u];
                    if (((t & k) == 0) ? (y < x) : (x < y)) {
                        keys[t] = y;
                        keys[u] = x;
                    }
                }
            }
            __syncthreads();
        }
    // 4b. conflict edges: pairs inside each run of equal vertex
    for (int t = tid; t < K; t += nt) {
        const unsigned long long kt = keys[t];
        const unsigned a = (unsigned)(kt & 0xFFFFu);
        for (int u = t + 1; u < K && (keys[u] >> 16) == (kt >> 16); u++) {
            const unsigned b = (unsigned)(keys[u] & 0xFFFFu);
            atomicOr(adj + (size_t)a * A.wcap + (b >> 5), 1u << (b & 31));
            atomicOr(adj + (size_t)b * A.wcap + (a >> 5), 1u << (a & 31));
        }
    }
    __syncthreads();
    if (tid == 0) A.n_inst[p] = N;
}

// Maximum independent set of one pattern's instances by branch and bound, one warp: a node holds
// the candidate set C (instances still compatible with the chosen ones) and the chosen count s.
// It is cut when s + |C| cannot beat the best set found; otherwise its first candidate v is
// taken (C minus v and its conflicts) and, unless v conflicts with nothing in C (then taking
// it is never worse), also left out (C minus v).  Nodes beyond the budget leave a lower bound.
__global__ void __launch_bounds__(32) k_exact_bb(ExactArgs A) {
    const int p = blockIdx.x, lane = threadIdx.x;
    const Plan &Q = A.plans[p];
    if (Q.status != FLEXIS_OK || !Q.exact_mis) return;
    flexis_support_result &R = A.results[p];
    const int N = A.n_inst[p];
    const long long lower = R.mis > 0 ? R.mis : 0;  // the greedy's maximal set is independent
    if (N < 0) {
        if (lane == 0) {
            R.mis_exact = lower;
            R.flags |= FLEXIS_FLAG_EXACT_MIS_SATURATED;
        }
        return;
    }
    const int W = (N + 31) / 32, WC = A.wcap;
    const uint32_t *adj = A.adj + (size_t)p * A.inst_cap * WC;
    uint32_t *frames = A.frames + (size_t)p * (A.inst_cap + 1) * WC;
    int32_t *meta = A.fmeta + (size_t)p * (A.inst_cap + 1) * 3;
    auto word_all = [&](int w) -> uint32_t {  // bits of instances 32w .. 32w+31 that exist
        const int lo = 32 * w;
        return N - lo >= 32 ? 0xFFFFFFFFu : (N > lo ? ((1u << (N - lo)) - 1u) : 0u);
    };
    for (int w = lane; w < W; w += 32) frames[w] = word_all(w);
    if (lane == 0) { meta[0] = 0; meta[1] = -1; meta[2] = 0; }
    __syncwarp();
    long long best = 0, nodes = 0;
    bool cut = false;
    int d = 0;
    while (d >= 0) {
        uint32_t *C = frames + (size_t)d * WC;
        const int size = meta[3 * d], state = meta[3 * d + 2];
        if (state == 0) {
            if (++nodes > A.node_budget) { cut = true; break; }
            int cnt = 0;
            for (int w = lane; w < W; w += 32) cnt += __popc(C[w]);
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULLMASK, cnt, o);
            if (size + cnt <= best) { d--; continue; }
            if (cnt == 0) { best = size; d--; continue; }
            // first candidate v
            int v = INT_MAX;
            for (int w = lane; w < W; w += 32)
                if (C[w]) { v = 32 * w + __ffs(C[w]) - 1; break; }
            for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULLMASK, v, o));
            const uint32_t *Nv = adj + (size_t)v * WC;
            bool conflicts = false;
            for (int w = lane; w < W; w += 32) conflicts |= (Nv[w] & C[w]) != 0u;
            conflicts = __any_sync(FULLMASK, conflicts);
            // child: take v
            uint32_t *D = frames + (size_t)(d + 1) * WC;
            for (int w = lane; w < W; w += 32) {
                uint32_t x = C[w] & ~Nv[w];
                if (w == (v >> 5)) x &= ~(1u << (v & 31));
                D[w] = x;
            }
            if (lane == 0) {
                meta[3 * d + 1] = v;
                meta[3 * d + 2] = conflicts ? 1 : 2;  // 1: leave-out branch still to do
                meta[3 * (d + 1)] = size + 1;
                meta[3 * (d + 1) + 2] = 0;
            }
            __syncwarp();
            d++;
        } else if (state == 1) {
            // child: leave v out
            const int v = meta[3 * d + 1];
            uint32_t *D = frames + (size_t)(d + 1) * WC;
            for (int w = lane; w < W; w += 32) {
                uint32_t x = C[w];
                if (w == (v >> 5)) x &= ~(1u << (v & 31));
                D[w] = x;
            }
            if (lane == 0) {
                meta[3 * d + 2] = 2;
                meta[3 * (d + 1)] = size;
                meta[3 * (d + 1) + 2] = 0;
            }
            __syncwarp();
            d++;
        } else {
            d--;
        }
    }
    if (lane == 0) {
        R.mis_exact = cut ? max(best, lower) : best;
        if (cut) R.flags |= FLEXIS_FLAG_EXACT_MIS_SATURATED;
    }
}

// ------------------------------------------------------------------ host driver
struct EnumWS {
    int64_t C = 0;     // rows per level buffer
    int32_t P = 0;     // pattern capacity
    int32_t maps_per = 0;
    int32_t *rows[MAXN] = {};                // level i rows (i >= 1): C * (i + 2) ints
    unsigned long long *off[MAXN] = {};      // level i counts, then their exclusive prefix (C + 1)
    unsigned long long *tsum = nullptr;      // scan tile sums
    unsigned long long *n_maps = nullptr;    // [P]
    unsigned long long *maps_n = nullptr;    // [P]
    unsigned long long *prefix = nullptr;    // [P + 1]
    unsigned long long *ctl = nullptr;       // [0] row counter, [1] split, [2..] stats
    unsigned long long *h_ctl = nullptr;     // pinned mirror (8 words)
    int32_t *maps = nullptr;                 // [P][maps_per][MAXN]
    // exact MIS (allocated when first needed): see ExactArgs
    int32_t xP = 0, x_inst = 0, x_maps = 0;
    int32_t last_inst_cap = 0;  // instance limit of the last exact-MIS pass (overlap read-back)
    int32_t *sidx = nullptr, *inst = nullptr, *n_inst = nullptr, *fmeta = nullptr;
    unsigned long long *keys = nullptr;
    uint32_t *adj = nullptr, *frames = nullptr;
    int64_t bytes = 0;
};

static int pow2_at_least(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return (int)p;
}

void enum_ws_destroy(DeviceGraph *g) {
    EnumWS *w = g->ews;
    if (!w) return;
    for (int i = 0; i < MAXN; i++) {
        cudaFree(w->rows[i]);
        cudaFree(w->off[i]);
    }
    cudaFree(w->tsum);
    cudaFree(w->n_maps);
    cudaFree(w->maps_n);
    cudaFree(w->prefix);
    cudaFree(w->ctl);
    cudaFree(w->maps);
    cudaFree(w->sidx); cudaFree(w->inst); cudaFree(w->n_inst); cudaFree(w->fmeta);
    cudaFree(w->keys); cudaFree(w->adj); cudaFree(w->frames);
    if (w->h_ctl) cudaFreeHost(w->h_ctl);
    delete w;
    g->ews = nullptr;
}

// buffers of the exact MIS for P patterns of at most inst_cap instances and maps_per maps
static int exact_ensure(EnumWS *w, int32_t P, int32_t inst_cap, int32_t maps_per) {
    if (w->sidx && w->xP >= P && w->x_inst >= inst_cap && w->x_maps >= maps_per) return FLEXIS_OK;
    P = std::max(P, w->xP);
    inst_cap = std::max(inst_cap, w->x_inst);
    maps_per = std::max(maps_per, w->x_maps);
    cudaFree(w->sidx); cudaFree(w->inst); cudaFree(w->n_inst); cudaFree(w->fmeta);
    cudaFree(w->keys); cudaFree(w->adj); cudaFree(w->frames);
    w->sidx = w->inst = w->n_inst = w->fmeta = nullptr;
    w->keys = nullptr;
    w->adj = w->frames = nullptr;
    w->xP = w->x_inst = w->x_maps = 0;
    const size_t wcap = (size_t)(inst_cap + 31) / 32;
    const size_t sp = (size_t)pow2_at_least(maps_per), kp = (size_t)pow2_at_least((int64_t)inst_cap * MAXN);
    CK(cudaMalloc((void **)&w->sidx, sizeof(int32_t) * P * sp));
    CK(cudaMalloc((void **)&w->inst, sizeof(int32_t) * P * inst_cap * MAXN));
    CK(cudaMalloc((void **)&w->n_inst, sizeof(int32_t) * P));
    CK(cudaMalloc((void **)&w->keys, sizeof(unsigned long long) * P * kp));
    CK(cudaMalloc((void **)&w->adj, sizeof(uint32_t) * P * inst_cap * wcap));
    CK(cudaMalloc((void **)&w->frames, sizeof(uint32_t) * P * (inst_cap + 1) * wcap));
    CK(cudaMalloc((void **)&w->fmeta, sizeof(int32_t) * P * (inst_cap + 1) * 3));
    w->xP = P;
    w->x_inst = inst_cap;
    w->x_maps = maps_per;
    return FLEXIS_OK;
}

static int enum_ws_ensure(DeviceGraph *g, int64_t C, int32_t P, int32_t maps_per) {
    EnumWS *w = g->ews;
    if (w && w->C >= C && w->P >= P && w->maps_per >= maps_per) return FLEXIS_OK;
    const int64_t nC = std::max(C, w ? w->C : 0);
    const int32_t nP = std::max(P, w ? w->P : 0);
    const int32_t nM = std::max(maps_per, w ? w->maps_per : 0);
    enum_ws_destroy(g);
    w = new EnumWS();
    g->ews = w;
    w->C = nC;
    w->P = nP;
    w->maps_per = nM;
    auto alloc = [&](void **p, size_t b) {
        w->bytes += (int64_t)b;
        return cudaMalloc(p, std::max<size_t>(b, 16));
    };
    // rows of levels 1 .. MAXN-2 (level MAXN-1 rows are final: counted, never written)
    for (int i = 1; i < MAXN - 1; i++) CK(alloc((void **)&w->rows[i], sizeof(int32_t) * (size_t)nC * (i + 2)));
    for (int i = 0; i < MAXN - 1; i++) CK(alloc((void **)&w->off[i], sizeof(unsigned long long) * (size_t)(nC + 2)));
    CK(alloc((void **)&w->tsum, sizeof(unsigned long long) * (size_t)((nC + 1) / SCAN_TILE + 2)));
    CK(alloc((void **)&w->n_maps, sizeof(unsigned long long) * (size_t)nP));
    CK(alloc((void **)&w->maps_n, sizeof(unsigned long long) * (size_t)nP));
    CK(alloc((void **)&w->prefix, sizeof(unsigned long long) * (size_t)(nP + 1)));
    CK(alloc((void **)&w->ctl, sizeof(unsigned long long) * 8));
    if (nM > 0) CK(alloc((void **)&w->maps, sizeof(int32_t) * (size_t)nP * nM * MAXN));
    CK(cudaMallocHost((void **)&w->h_ctl, sizeof(unsigned long long) * 8));
    return FLEXIS_OK;
}

namespace {

struct EnumRun {
    DeviceGraph *g;
    EnumWS *w;
    EnumPass E;       // fields common to every launch
    cudaStream_t s;
    int blocks;
    std::chrono::steady_clock::time_point t0;
    int32_t deadline_ms;
    bool timed_out = false;
    int64_t launches = 0;

    bool past() {
        if (deadline_ms <= 0) return false;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > deadline_ms) timed_out = true;
        return timed_out;
    }

    int scan(unsigned long long *cnt_off, long long n) {
        launches += 3;
        return dev_scan_u64(cnt_off, n, w->tsum, s);
    }

    // read one device word (synchronises the stream)
    int read(const unsigned long long *d, unsigned long long *h) {
        CK(cudaMemcpyAsync(w->h_ctl, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *h = w->h_ctl[0];
        return FLEXIS_OK;
    }

    // Process rows [0, nrows) of level `level` (level 0: virtual roots).
    int level(int lv, long long nrows) {
        const int64_t C = w->C;
        for (long long a = 0; a < nrows; a += C) {
            if (past()) return FLEXIS_OK;
            const long long n = std::min<long long>(C, nrows - a);
            EnumPass e = E;
            e.level = lv;
            e.in = lv > 0 ? w->rows[lv] : nullptr;
            e.row0 = a;
            e.nrows = n;
            e.cnt = w->off[lv];
            CK(cudaMemsetAsync(w->ctl, 0, sizeof(unsigned long long), s));
            k_extend<false><<<blocks, ENUM_THREADS, 0, s>>>(e);
            launches++;
            CK(cudaGetLastError());
            if (lv + 1 >= MAXN - 1) continue;  // level MAXN-1 rows are always final
            int rc = scan(w->off[lv], n);
            if (rc) return rc;
            unsigned long long total = 0;
            if ((rc = read(w->off[lv] + n, &total))) return rc;
            if (total == 0) continue;
            long long pos = 0;
            while (pos < n) {
                if (past()) return FLEXIS_OK;
                k_split<<<1, 1, 0, s>>>(w->off[lv], pos, n, (unsigned long long)C, w->ctl + 1);
                launches++;
                unsigned long long end = 0;
                if ((rc = read(w->ctl + 1, &end))) return rc;
                unsigned long long opos = 0, oend = 0;
                CK(cudaMemcpyAsync(w->h_ctl, w->off[lv] + pos, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(w->h_ctl + 1, w->off[lv] + end, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                opos = w->h_ctl[0];
                oend = w->h_ctl[1];
                if (oend > opos) {
                    EnumPass f = E;
                    f.level = lv;
                    f.in = lv > 0 ? w->rows[lv] : nullptr;
                    f.row0 = a + pos;
                    f.nrows = (long long)end - pos;
                    f.off = w->off[lv] + pos;
                    f.out = w->rows[lv + 1];
                    CK(cudaMemsetAsync(w->ctl, 0, sizeof(unsigned long long), s));
                    k_extend<true><<<blocks, ENUM_THREADS, 0, s>>>(f);
                    launches++;
                    CK(cudaGetLastError());
                    if ((rc = level(lv + 1, (long long)(oend - opos)))) return rc;
                    if (timed_out) return FLEXIS_OK;
                }
                pos = (long long)end;
            }
        }
        return FLEXIS_OK;
    }
};

}  // namespace

int dev_enumerate(DeviceGraph *g, const Plan *d_plans, int32_t P, flexis_support_result *d_results,
                  cudaStream_t stream, const EvalConfig &cfg, flexis_stats *stats,
                  std::chrono::steady_clock::time_point t_start) {
    if (P <= 0) return FLEXIS_OK;
    const int64_t C = std::max<int64_t>(cfg.frontier_rows > 0 ? cfg.frontier_rows : ENUM_DEFAULT_ROWS,
                                        (int64_t)g->max_degree + 64);
    const int32_t maps_per = cfg.exact_mis ? cfg.exact_mis_maps_buffer : 0;
    int rc = enum_ws_ensure(g, C, P, maps_per);
    if (rc) return rc;
    EnumWS *w = g->ews;
    EnumRun R;
    R.g = g;
    R.w = w;
    R.s = stream;
    R.t0 = t_start;
    R.deadline_ms = cfg.deadline_ms;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_extend<false>, ENUM_THREADS, 0) != cudaSuccess)
        per_sm = 1;
    R.blocks = g->sm_count * std::max(1, per_sm);
    EnumPass &E = R.E;
    memset(&E, 0, sizeof E);
    E.G = g->view;
    E.plans = d_plans;
    E.P = P;
    E.root_prefix = w->prefix;
    E.n_maps = w->n_maps;
    E.maps_cap = cfg.maps_cap > 0 ? (unsigned long long)cfg.maps_cap : DEFAULT_MAPS_CAP;
    E.maps = maps_per > 0 ? w->maps : nullptr;
    E.maps_n = w->maps_n;
    E.maps_per = maps_per;
    E.next = w->ctl;
    E.stat = w->ctl + 2;
    CK(cudaMemsetAsync(w->n_maps, 0, sizeof(unsigned long long) * P, stream));
    CK(cudaMemsetAsync(w->maps_n, 0, sizeof(unsigned long long) * P, stream));
    CK(cudaMemsetAsync(w->ctl, 0, sizeof(unsigned long long) * 8, stream));
    k_enum_prefix<<<1, 1024, 0, stream>>>(d_plans, P, w->prefix);
    R.launches++;
    CK(cudaGetLastError());
    unsigned long long roots = 0;
    rc = R.read(w->prefix + P, &roots);
    if (rc) return rc;
    if (roots > 0) {
        rc = R.level(0, (long long)roots);
        if (rc) return rc;
    }
    if (maps_per > 0 && !R.timed_out) {
        const int32_t inst_cap = std::max(1, cfg.exact_mis_maps);
        if ((rc = exact_ensure(w, P, inst_cap, maps_per))) return rc;
        ExactArgs A;
        memset(&A, 0, sizeof A);
        A.plans = d_plans;
        A.P = P;
        A.maps = w->maps;
        A.maps_n = w->maps_n;
        A.maps_per = maps_per;
        A.inst_cap = inst_cap;
        A.wcap = (inst_cap + 31) / 32;
        A.sidx_stride = pow2_at_least(w->x_maps);
        A.keys_stride = pow2_at_least((int64_t)w->x_inst * MAXN);
        A.sidx = w->sidx;
        A.inst = w->inst;
        A.n_inst = w->n_inst;
        A.keys = w->keys;
        A.adj = w->adj;
        A.frames = w->frames;
        A.fmeta = w->fmeta;
        A.node_budget = cfg.exact_mis_nodes > 0 ? cfg.exact_mis_nodes : (1ll << 24);
        A.results = d_results;
        w->last_inst_cap = inst_cap;
        k_exact_prepare<<<P, 1024, 0, stream>>>(A);
        k_exact_bb<<<P, 32, 0, stream>>>(A);
        R.launches += 2;
        CK(cudaGetLastError());
    }
    k_enum_finalize<<<(P + 255) / 256, 256, 0, stream>>>(d_plans, P, d_results, w->n_maps, E.maps_cap,
                                                         R.timed_out ? 1 : 0);
    R.launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(w->h_ctl, w->ctl, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (stats) {
        stats->kernel_launches += R.launches;
        stats->enum_rows += (int64_t)w->h_ctl[2 + EST_ROWS];
        stats->enum_scanned += (int64_t)w->h_ctl[2 + EST_SCANNED];
        stats->enum_bytes += (int64_t)w->h_ctl[2 + EST_BYTES];
    }
    return FLEXIS_OK;  // a deadline shows in the patterns' status (k_enum_finalize)
}

}  // namespace fx

namespace fx {

int dev_overlap_read(DeviceGraph *g, int32_t p, int32_t *inst_out, int64_t cap_inst, int64_t *n_inst,
                     int32_t *edges_out, int64_t cap_edges, int64_t *n_edges) {
    EnumWS *w = g->ews;
    if (!w || !w->n_inst || p < 0 || p >= w->xP || w->last_inst_cap <= 0) return FLEXIS_E_INVALID;
    CK(cudaSetDevice(g->device));
    int32_t N = 0;
    CK(cudaMemcpy(&N, w->n_inst + p, sizeof N, cudaMemcpyDeviceToHost));
    *n_inst = N;
    *n_edges = 0;
    if (N < 0) return FLEXIS_E_UNSUPPORTED;  // more maps or instances than the limits
    const int inst_cap = w->last_inst_cap, wcap = (inst_cap + 31) / 32;
    std::vector<int32_t> inst((size_t)N * MAXN);
    std::vector<uint32_t> adj((size_t)N * wcap);
    if (N > 0) {
        CK(cudaMemcpy(inst.data(), w->inst + (size_t)p * inst_cap * MAXN, sizeof(int32_t) * inst.size(),
                      cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(adj.data(), w->adj + (size_t)p * inst_cap * wcap, sizeof(uint32_t) * adj.size(),
                      cudaMemcpyDeviceToHost));
    }
    for (int64_t i = 0; i < std::min<int64_t>(N, cap_inst) * MAXN; i++) inst_out[i] = inst[(size_t)i];
    int64_t e = 0;
    for (int32_t a = 0; a < N; a++)
        for (int32_t b = a + 1; b < N; b++)
            if (adj[(size_t)a * wcap + (b >> 5)] >> (b & 31) & 1u) {
                if (e < cap_edges) {
                    edges_out[2 * e] = a;
                    edges_out[2 * e + 1] = b;
                }
                e++;
            }
    *n_edges = e;
    return FLEXIS_OK;
}

}  // namespace fx
