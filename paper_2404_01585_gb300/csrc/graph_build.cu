// Device construction of the resident undirected data-graph layout.
//
// Builds, from the caller's edge list, the four arrays of the host builder (graph.cpp) bit for
// bit: per vertex the adjacency sorted by (label rank, id) without repeats, the label runs with
// a sentinel, one 32-byte record, and the label-partitioned vertex index in greedy-root order.
// A graph therefore evaluates identically whichever side built it.  The host keeps only the
// label tables (ranks by ascending frequency, ties by id; vertices per rank), which take one
// pass over the labels.
//
// With A = 2 x edges arcs:
//   1. k_gb_arcs: edge e gives the arcs 2e = (src, dst) and 2e + 1 = (dst, src), each packed as
//      (v << 32 | w).  A self-loop's arcs get v = nv, a row past the last vertex, so they sort to
//      the end and are dropped there.  An endpoint out of range is counted (FLEXIS_E_INVALID).
//   2. a stable least-significant-digit radix sort of the arcs, 8 bits a pass, by
//      (v, rank(w), w): passes over the bytes of w, then over rank(w), then over the bytes of v.
//      A pass is a per-tile digit histogram, one exclusive scan of the histograms laid out
//      digit-major (giving every (digit, tile) its output base), and a scatter that keeps the
//      input order among equal digits: ranks inside a warp come from __match_any_sync, and a
//      running per-digit offset orders the warps of a tile and its rounds.
//   3. k_gb_mark: an arc is kept if v < nv and it differs from its predecessor (repeats are
//      adjacent after the sort).  A kept arc opens a label run if its predecessor lies in another
//      row or has another neighbour rank.  Per arc the flag word (opens-run << 32 | kept); per
//      row one atomic add of that word (runs << 32 | degree), the neighbour-rank mask and the
//      label pairs present (both from run openers only: a run has one neighbour rank).
//   4. two exclusive scans: of the flag words over the arcs (adjacency position, run index) and
//      of the row words over the vertices (row offsets).  The low halves never carry into the
//      high halves because A < 2^32.
//   5. k_gb_write: adjacency and run entries; k_gb_rows: each vertex's sentinel run and record.
//   6. lab_vtx: vertex ids radix-sorted by the 8 bytes of H(seed, v) (no pass for the id order),
//      then by rank.  From the identity order, stable passes give (rank, H(seed, v), v).
#include <algorithm>
#include <cstring>
#include <vector>

#include "fx_kern.cuh"

namespace fx {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr long long RS_TILE = (long long)RS_THREADS * RS_ITEMS;
constexpr int GB_THREADS = 256;

enum { DIG_LO = 0, DIG_RANK = 1, DIG_HI = 2, DIG_HASH = 3 };
enum { GB_BAD = 0, GB_LOOPS = 1, GB_MAXDEG = 2, GB_CTL = 4 };

struct RadixPass {
    const unsigned long long *in;
    unsigned long long *out;
    long long n;
    int tiles;
    int mode;   // DIG_*: which byte of the element is the digit
    int shift;  // bit offset of that byte
    const uint8_t *rk;
    unsigned long long seed;
    unsigned long long *hist;  // [256 * tiles + 1]: digit-major counts, then their exclusive scan
};

// H(seed, v): one SplitMix64 step (Steele, Lea, Flood 2014) from state seed XOR v, the same
// greedy-order key the host builder sorts by.
__device__ __forceinline__ unsigned long long order_hash(unsigned long long seed, unsigned long long v) {
    unsigned long long z = (seed ^ v) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int digit_of(const RadixPass &R, unsigned long long x) {
    const uint32_t lo = (uint32_t)x;
    switch (R.mode) {
        case DIG_LO: return (int)((lo >> R.shift) & 0xFFu);
        case DIG_RANK: return (int)__ldg(R.rk + lo);
        case DIG_HI: return (int)(((uint32_t)(x >> 32) >> R.shift) & 0xFFu);
        default: return (int)((order_hash(R.seed, lo) >> R.shift) & 0xFFull);
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(RadixPass R) {
    __shared__ unsigned int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; r++) {
        const long long i = base + (long long)r * RS_THREADS + threadIdx.x;
        if (i < R.n) atomicAdd(&cnt[digit_of(R, R.in[i])], 1u);
    }
    __syncthreads();
    R.hist[(long long)threadIdx.x * R.tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile: element base + r * 256 + t is handled in round r by thread t, so
// rounds, then warps, then lanes follow the input order.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(RadixPass R) {
    __shared__ unsigned int run[256];           // next output position per digit (thread d owns d)
    __shared__ unsigned int wc[RS_WARPS][256];  // per round: warp counts, then warp bases
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = (unsigned int)R.hist[(long long)tid * R.tiles + blockIdx.x];
    const long long base = (long long)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; r++) {
        if (base + (long long)r * RS_THREADS >= R.n) break;  // the same for every thread
        const long long i = base + (long long)r * RS_THREADS + tid;
        const bool valid = i < R.n;
        unsigned long long x = 0;
        int d = 256;
        if (valid) {
            x = R.in[i];
            d = digit_of(R, x);
        }
        for (int k = tid; k < RS_WARPS * 256; k += RS_THREADS) (&wc[0][0])[k] = 0;
        __syncthreads();
        const unsigned int m = __match_any_sync(FULLMASK, d);
        const int lr = __popc(m & ((1u << lane) - 1u));
        if (valid && lr == 0) wc[warp][d] = (unsigned int)__popc(m);
        __syncthreads();
        unsigned int s = run[tid];
        for (int w = 0; w < RS_WARPS; w++) {
            const unsigned int c = wc[w][tid];
            wc[w][tid] = s;
            s += c;
        }
        run[tid] = s;
        __syncthreads();
        if (valid) R.out[wc[warp][d] + (unsigned int)lr] = x;
        __syncthreads();
    }
}

__global__ void k_gb_arcs(const int32_t *src, const int32_t *dst, long long ne, long long nv,
                          unsigned long long *arcs, unsigned long long *ctl) {
    unsigned long long bad = 0, loops = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        long long a = src[e], b = dst[e];
        if (a < 0 || b < 0 || a >= nv || b >= nv) {
            bad++;
            a = b = 0;  // kept in range; the load fails
        } else if (a == b) {
            loops++;
        }
        const unsigned long long va = a == b ? (unsigned long long)nv : (unsigned long long)a;
        const unsigned long long vb = a == b ? (unsigned long long)nv : (unsigned long long)b;
        arcs[2 * e] = va << 32 | (unsigned long long)(uint32_t)b;
        arcs[2 * e + 1] = vb << 32 | (unsigned long long)(uint32_t)a;
    }
    bad = __reduce_add_sync(FULLMASK, (unsigned int)bad);
    loops = __reduce_add_sync(FULLMASK, (unsigned int)loops);
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(&ctl[GB_BAD], bad);
        if (loops) atomicAdd(&ctl[GB_LOOPS], loops);
    }
}

__global__ void k_gb_mark(const unsigned long long *arcs, long long A, long long nv, const uint8_t *rk, int nl,
                          unsigned long long *flags, unsigned long long *rowc, unsigned long long *lm,
                          unsigned int *pairs) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long x = arcs[i];
        const long long v = (long long)(x >> 32);
        unsigned long long f = 0;
        if (v < nv) {
            const unsigned long long p = i > 0 ? arcs[i - 1] : ~0ull;
            if (p != x) {
                const uint32_t w = (uint32_t)x;
                const int rw = rk[w];
                const bool opens = i == 0 || (long long)(p >> 32) != v || rk[(uint32_t)p] != rw;
                f = (opens ? 1ull << 32 : 0ull) | 1ull;
                atomicAdd(&rowc[v], f);
                if (opens) {
                    if (rw < 64) atomicOr(&lm[v], 1ull << rw);
                    const int rv = rk[v];
                    if (rv <= rw) pairs[rv * nl + rw] = 1u;
                }
            }
        }
        flags[i] = f;
    }
}

__global__ void k_gb_write(const unsigned long long *arcs, long long A, const uint8_t *rk,
                           const unsigned long long *flags, const unsigned long long *rows, int32_t *adj,
                           uint32_t *runs) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long f0 = flags[i], f1 = flags[i + 1];
        if (f1 == f0) continue;  // not kept
        const unsigned long long x = arcs[i];
        const uint32_t v = (uint32_t)(x >> 32), w = (uint32_t)x;
        const uint32_t pos = (uint32_t)f0;
        adj[pos] = (int32_t)w;
        if ((f1 >> 32) != (f0 >> 32))
            runs[(f0 >> 32) + v] = (uint32_t)rk[w] << 24 | (pos - (uint32_t)rows[v]);
    }
}

__global__ void k_gb_rows(long long nv, const uint8_t *rk, const unsigned long long *rows, const unsigned long long *lm,
                          uint32_t *runs, VRec *vrec, unsigned long long *ctl) {
    unsigned int dmax = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        const unsigned long long r0 = rows[v], r1 = rows[v + 1];
        const uint32_t deg = (uint32_t)r1 - (uint32_t)r0;
        const uint32_t nrun = (uint32_t)(r1 >> 32) - (uint32_t)(r0 >> 32);
        const uint32_t roff = (uint32_t)(r0 >> 32) + (uint32_t)v;
        runs[roff + nrun] = RUN_SENTINEL_LABEL << 24 | deg;
        VRec rec;
        rec.adj = (uint32_t)r0;
        rec.run = roff;
        rec.deg = deg;
        rec.meta = nrun << 8 | (uint32_t)rk[v];
        rec.nbr_labels = lm[v];
        rec.pad = 0;
        vrec[v] = rec;
        dmax = max(dmax, deg);
    }
    dmax = __reduce_max_sync(FULLMASK, dmax);
    if ((threadIdx.x & 31) == 0 && dmax) atomicMax(&ctl[GB_MAXDEG], (unsigned long long)dmax);
}

__global__ void k_gb_iota(unsigned long long *a, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = (unsigned long long)i;
}

__global__ void k_gb_low(const unsigned long long *a, long long n, int32_t *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (int32_t)(uint32_t)a[i];
}

namespace {

// Device temporaries of one build, freed on every exit.
struct Temps {
    std::vector<void *> p;
    int get(void **out, size_t bytes) {
        *out = nullptr;
        if (cudaMalloc(out, std::max<size_t>(bytes, 16)) != cudaSuccess) return FLEXIS_E_NOMEM;
        p.push_back(*out);
        return FLEXIS_OK;
    }
    ~Temps() {
        for (void *q : p) cudaFree(q);
    }
};

int bit_width(unsigned long long x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

struct Sorter {
    cudaStream_t s;
    unsigned long long *hist, *tsum;
    const uint8_t *rk;
    unsigned long long seed;

    // One stable pass from *a into *b, then the two swapped.
    int pass(unsigned long long **a, unsigned long long **b, long long n, int mode, int shift) {
        if (n == 0) return FLEXIS_OK;
        RadixPass R;
        R.in = *a;
        R.out = *b;
        R.n = n;
        R.tiles = (int)((n + RS_TILE - 1) / RS_TILE);
        R.mode = mode;
        R.shift = shift;
        R.rk = rk;
        R.seed = seed;
        R.hist = hist;
        k_rs_hist<<<R.tiles, RS_THREADS, 0, s>>>(R);
        CK(cudaGetLastError());
        const int rc = dev_scan_u64(hist, 256ll * R.tiles, tsum, s);
        if (rc) return rc;
        k_rs_scatter<<<R.tiles, RS_THREADS, 0, s>>>(R);
        CK(cudaGetLastError());
        std::swap(*a, *b);
        return FLEXIS_OK;
    }
};

int grid_for(long long n, int sm_count) {
    const long long want = (n + GB_THREADS - 1) / GB_THREADS;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)sm_count * 8));
}

}  // namespace

int dev_graph_build(int64_t nv, const int32_t *labels, int64_t ne, const int32_t *src, const int32_t *dst,
                    uint64_t seed, int id_order, int device, HostGraph &hg, DeviceGraph **out) {
    if (nv < 0 || ne < 0 || (nv > 0 && !labels) || (ne > 0 && (!src || !dst))) return FLEXIS_E_INVALID;
    if (nv >= (int64_t)INT32_MAX) return FLEXIS_E_UNSUPPORTED;
    hg = HostGraph();
    hg.nv = nv;
    hg.seed = seed;
    for (int64_t v = 0; v < nv; v++)
        if (labels[v] < 0) return FLEXIS_E_INVALID;
    // label tables on the host; a failure here is reported after the edge check, as the host
    // builder orders them
    std::vector<uint8_t> rk;
    const int label_rc = label_ranks(nv, labels, hg, rk);
    if (label_rc == FLEXIS_E_INVALID) return label_rc;

    DeviceGraph *g = nullptr;
    int rc = dev_graph_init(device, &g);
    if (rc) return rc;
    auto fail = [&](int code) {
        dev_graph_destroy(g);
        return code;
    };
    const cudaStream_t s = g->stream;
    const long long A = 2 * (long long)ne;
    const long long nvl = nv;
    Temps T;
    unsigned long long *arcs = nullptr, *arcs2 = nullptr, *flags = nullptr, *rowc = nullptr, *lm = nullptr;
    unsigned long long *hist = nullptr, *tsum = nullptr, *ctl = nullptr;
    int32_t *d_src = nullptr, *d_dst = nullptr;
    uint8_t *d_rk = nullptr;
    unsigned int *pairs = nullptr;
    const long long nl2 = std::max<long long>(1, (long long)hg.nl * hg.nl);
    const long long sortn = std::max<long long>(A, nvl);
    const long long hist_n = 256ll * ((sortn + RS_TILE - 1) / RS_TILE);
    const long long scan_n = std::max<long long>(std::max(hist_n, A + 1), nvl + 1);
    if (T.get((void **)&arcs, 8 * (size_t)sortn) || T.get((void **)&arcs2, 8 * (size_t)sortn) ||
        T.get((void **)&flags, 8 * (size_t)(A + 1)) || T.get((void **)&rowc, 8 * (size_t)(nvl + 1)) ||
        T.get((void **)&lm, 8 * (size_t)std::max<long long>(nvl, 1)) ||
        T.get((void **)&hist, 8 * (size_t)(hist_n + 1)) ||
        T.get((void **)&tsum, 8 * (size_t)scan_tsum_len(scan_n)) || T.get((void **)&ctl, 8 * GB_CTL) ||
        T.get((void **)&d_src, 4 * (size_t)ne) || T.get((void **)&d_dst, 4 * (size_t)ne) ||
        T.get((void **)&d_rk, (size_t)std::max<long long>(nvl, 1)) || T.get((void **)&pairs, 4 * (size_t)nl2))
        return fail(FLEXIS_E_NOMEM);
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaMemsetAsync(ctl, 0, 8 * GB_CTL, s)) || !ok(cudaMemsetAsync(rowc, 0, 8 * (size_t)(nvl + 1), s)) ||
        !ok(cudaMemsetAsync(lm, 0, 8 * (size_t)std::max<long long>(nvl, 1), s)) ||
        !ok(cudaMemsetAsync(pairs, 0, 4 * (size_t)nl2, s)))
        return fail(FLEXIS_E_CUDA);
    if (ne > 0 && (!ok(cudaMemcpyAsync(d_src, src, 4 * (size_t)ne, cudaMemcpyHostToDevice, s)) ||
                   !ok(cudaMemcpyAsync(d_dst, dst, 4 * (size_t)ne, cudaMemcpyHostToDevice, s))))
        return fail(FLEXIS_E_CUDA);
    const int sm = std::max(1, g->sm_count);
    // 1: arcs (and the endpoint check)
    if (A > 0) {
        k_gb_arcs<<<grid_for(ne, sm), GB_THREADS, 0, s>>>(d_src, d_dst, ne, nvl, arcs, ctl);
        if (!ok(cudaGetLastError())) return fail(FLEXIS_E_CUDA);
    }
    if (label_rc) {  // too many labels: no layout, but a bad endpoint is reported first
        unsigned long long bad = 0;
        if (!ok(cudaMemcpyAsync(&bad, ctl + GB_BAD, 8, cudaMemcpyDeviceToHost, s)) || !ok(cudaStreamSynchronize(s)))
            return fail(FLEXIS_E_CUDA);
        return fail(bad ? FLEXIS_E_INVALID : label_rc);
    }
    if (!ok(cudaMemcpyAsync(d_rk, rk.data(), (size_t)std::max<long long>(nvl, 1), cudaMemcpyHostToDevice, s)))
        return fail(FLEXIS_E_CUDA);
    g->upload_bytes = (int64_t)std::max<long long>(nvl, 1) + 8 * ne;

    // 2: arcs sorted by (v, rank(w), w)
    Sorter S{s, hist, tsum, d_rk, (unsigned long long)seed};
    if (A > 0) {
        const int wbits = bit_width((unsigned long long)std::max<long long>(nvl - 1, 0));
        const int vbits = bit_width((unsigned long long)nvl);
        for (int sh = 0; sh < wbits; sh += 8)
            if ((rc = S.pass(&arcs, &arcs2, A, DIG_LO, sh))) return fail(rc);
        if ((rc = S.pass(&arcs, &arcs2, A, DIG_RANK, 0))) return fail(rc);
        for (int sh = 0; sh < vbits; sh += 8)
            if ((rc = S.pass(&arcs, &arcs2, A, DIG_HI, sh))) return fail(rc);
        // 3-4: kept arcs, run openers, per-row words; scans
        k_gb_mark<<<grid_for(A, sm), GB_THREADS, 0, s>>>(arcs, A, nvl, d_rk, hg.nl, flags, rowc, lm, pairs);
        if (!ok(cudaGetLastError())) return fail(FLEXIS_E_CUDA);
    }
    if ((rc = dev_scan_u64(flags, A, tsum, s))) return fail(rc);
    if ((rc = dev_scan_u64(rowc, nvl, tsum, s))) return fail(rc);
    unsigned long long h[GB_CTL + 2];
    if (!ok(cudaMemcpyAsync(h, ctl, 8 * GB_CTL, cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaMemcpyAsync(h + GB_CTL, flags + A, 8, cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaMemcpyAsync(h + GB_CTL + 1, rowc + nvl, 8, cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaStreamSynchronize(s)))
        return fail(FLEXIS_E_CUDA);
    if (h[GB_BAD]) return fail(FLEXIS_E_INVALID);
    const unsigned long long tot = h[GB_CTL];
    if (tot != h[GB_CTL + 1]) return fail(FLEXIS_E_CUDA);  // the two scans count the same arcs
    const long long arcs_kept = (long long)(uint32_t)tot, openers = (long long)(tot >> 32);
    const long long nruns = openers + nvl;
    if (arcs_kept >= (long long)UINT32_MAX || nruns >= (long long)UINT32_MAX) return fail(FLEXIS_E_UNSUPPORTED);
    hg.self_loops = (int64_t)h[GB_LOOPS];
    hg.n_arcs = arcs_kept;
    hg.duplicates = (2 * (ne - hg.self_loops) - arcs_kept) / 2;

    // 5: the resident arrays (sizes as the host builder's, zero padded)
    const size_t b_vrec = sizeof(VRec) * (size_t)std::max<long long>(nvl, 1);
    const size_t b_runs = 4 * (size_t)std::max<long long>(nruns, 1);
    const size_t b_adj = 4 * (size_t)std::max<long long>(arcs_kept, 1);
    const size_t b_lab = 4 * (size_t)std::max<long long>(nvl, 1);
    if (!ok(cudaMalloc(&g->d_vrec, b_vrec)) || !ok(cudaMalloc(&g->d_runs, b_runs)) ||
        !ok(cudaMalloc(&g->d_adj, b_adj)) || !ok(cudaMalloc(&g->d_labvtx, b_lab)))
        return fail(FLEXIS_E_NOMEM);
    g->bytes = (int64_t)(b_vrec + b_runs + b_adj + b_lab);
    if (!ok(cudaMemsetAsync(g->d_vrec, 0, b_vrec, s)) || !ok(cudaMemsetAsync(g->d_runs, 0, b_runs, s)) ||
        !ok(cudaMemsetAsync(g->d_adj, 0, b_adj, s)) || !ok(cudaMemsetAsync(g->d_labvtx, 0, b_lab, s)))
        return fail(FLEXIS_E_CUDA);
    if (A > 0)
        k_gb_write<<<grid_for(A, sm), GB_THREADS, 0, s>>>(arcs, A, d_rk, flags, rowc, (int32_t *)g->d_adj,
                                                           (uint32_t *)g->d_runs);
    if (nvl > 0)
        k_gb_rows<<<grid_for(nvl, sm), GB_THREADS, 0, s>>>(nvl, d_rk, rowc, lm, (uint32_t *)g->d_runs,
                                                            (VRec *)g->d_vrec, ctl);
    if (!ok(cudaGetLastError())) return fail(FLEXIS_E_CUDA);

    // 6: lab_vtx
    if (nvl > 0) {
        k_gb_iota<<<grid_for(nvl, sm), GB_THREADS, 0, s>>>(arcs, nvl);
        if (!ok(cudaGetLastError())) return fail(FLEXIS_E_CUDA);
        if (!id_order)
            for (int sh = 0; sh < 64; sh += 8)
                if ((rc = S.pass(&arcs, &arcs2, nvl, DIG_HASH, sh))) return fail(rc);
        if ((rc = S.pass(&arcs, &arcs2, nvl, DIG_RANK, 0))) return fail(rc);
        k_gb_low<<<grid_for(nvl, sm), GB_THREADS, 0, s>>>(arcs, nvl, (int32_t *)g->d_labvtx);
        if (!ok(cudaGetLastError())) return fail(FLEXIS_E_CUDA);
    }
    std::vector<unsigned int> hp((size_t)nl2);
    if (!ok(cudaMemcpyAsync(h, ctl, 8 * GB_CTL, cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaMemcpyAsync(hp.data(), pairs, 4 * (size_t)nl2, cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaStreamSynchronize(s)))
        return fail(FLEXIS_E_CUDA);
    hg.max_degree = (int32_t)std::min<unsigned long long>(h[GB_MAXDEG], INT32_MAX);
    if (hg.max_degree >= (1 << 24)) return fail(FLEXIS_E_UNSUPPORTED);
    for (int a = 0; a < hg.nl; a++)
        for (int b = a; b < hg.nl; b++)
            if (hp[(size_t)a * (size_t)hg.nl + (size_t)b]) hg.label_pairs.emplace_back(a, b);

    g->built_on_device = 1;
    g->vrec_count = (int64_t)(b_vrec / sizeof(VRec));
    g->runs_words = (int64_t)(b_runs / 4);
    g->adj_words = (int64_t)(b_adj / 4);
    g->labvtx_words = (int64_t)(b_lab / 4);
    g->view.vrec = (const VRec *)g->d_vrec;
    g->view.runs = (const uint32_t *)g->d_runs;
    g->view.adj = (const int32_t *)g->d_adj;
    g->view.lab_vtx = (const int32_t *)g->d_labvtx;
    g->view.nv = nv;
    g->view.words = (int32_t)std::max<int64_t>(1, (nv + 31) / 32);
    g->view.dstride = 0;
    g->max_degree = hg.max_degree;
    *out = g;
    return FLEXIS_OK;
}

}  // namespace fx
