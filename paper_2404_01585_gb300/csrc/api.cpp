// C ABI of the FLEXIS GB300 library (declared in include/flexis.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "fx_dev.h"

using namespace fx;

struct flexis_graph {
    HostGraph hg;
    DeviceGraph *dg = nullptr;
    flexis_options opt{};
    flexis_stats last{};
    int64_t n_input_vertices = 0;  // vertices the caller passed
    int32_t edge_label_base = -1;  // label of edge label 0 in the extended graph; -1: none
    int64_t input_self_loops = 0, input_duplicates = 0;  // of the caller's edge list
    std::map<int, int32_t> tuned_budget;  // autotuner: per-round search budget per batch-size bucket
};

struct flexis_pattern_set {
    struct Entry {
        Code code;  // rank-space canonical code
        flexis_support_result res;
    };
    std::vector<Entry> items;
    std::vector<int32_t> label_of_rank;
    int64_t cand[FLEXIS_MAX_PATTERN + 1] = {0};
    int64_t freq[FLEXIS_MAX_PATTERN + 1] = {0};
};

namespace {

constexpr int64_t LAMBDA_DEN = FLEXIS_LAMBDA_DEN;

bool lambda_to_q(double lambda, int64_t *num) {
    if (!(lambda >= 0.0 && lambda <= 1.0)) return false;  // also rejects NaN
    *num = llround(lambda * (double)LAMBDA_DEN);
    return true;
}

using Clock = std::chrono::steady_clock;

float ms_since(Clock::time_point t0) {
    return std::chrono::duration<float, std::milli>(Clock::now() - t0).count();
}

int host_threads() { return (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency())); }

template <class F>
void parallel_chunks(int64_t n, int T, F f) {
    if (n < 256) T = 1;
    std::vector<std::thread> th;
    const int64_t chunk = (n + T - 1) / T;
    for (int t = 1; t < T; t++) {
        const int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
        if (lo < hi) th.emplace_back([=] { f(lo, hi); });
    }
    f(0, std::min(n, chunk));
    for (auto &x : th) x.join();
}

void add_stats(flexis_stats &a, const flexis_stats &b) {
    a.rounds += b.rounds;
    a.search_items += b.search_items;
    a.mni_items += b.mni_items;
    a.kernel_launches += b.kernel_launches;
    a.alg_bytes += b.alg_bytes;
    a.alg_bytes_greedy += b.alg_bytes_greedy;
    a.patterns += b.patterns;
    a.search_ms += b.search_ms;
    a.mni_ms += b.mni_ms;
    a.total_ms += b.total_ms;
    a.host_gen_ms += b.host_gen_ms;
    a.host_compile_ms += b.host_compile_ms;
    a.search_launches += b.search_launches;
    a.batches += b.batches;
    a.graph_launches += b.graph_launches;
    a.enum_rows += b.enum_rows;
    a.enum_scanned += b.enum_scanned;
    a.enum_bytes += b.enum_bytes;
    a.search_scanned += b.search_scanned;
    a.search_bound += b.search_bound;
    a.search_map_words += b.search_map_words;
    a.autotune_probes += b.autotune_probes;
    if (b.search_budget) a.search_budget = b.search_budget;
}

// Autotuner of the launch shape, by batch size: many patterns -> small windows (parallelism
// comes from the batch, and per-pattern window memory stays small); few patterns -> large
// windows (parallelism has to come from speculation inside each pattern).  Few patterns also
// get a small per-round search budget, so that heavy searches are split early and spread
// over the idle warps; a large batch already fills the GPU and keeps the default.
constexpr int32_t SMALL_BATCH = 1024, SMALL_BATCH_BUDGET = 256;

EvalConfig config_for(const flexis_graph *g, int32_t P) {
    EvalConfig c;
    int wmax = P < 64 ? 8192 : P < 4096 ? 4096 : P < 65536 ? 1024 : 512;
    int wmin = std::max(16, std::min(wmax, 16384 / std::max(1, P)));
    if (g->opt.window_max > 0) wmax = g->opt.window_max;
    if (g->opt.window_min > 0) wmin = g->opt.window_min;
    c.w_min = std::min(wmin, wmax);
    c.w_max = wmax;
    c.search_blocks = g->opt.search_blocks;
    c.record_selected = g->opt.record_selected;
    c.rounds_per_sync = P >= 64 ? 4 : 2;
    c.timing = g->opt.timing != 0;
    c.graphs = g->opt.graphs >= 0;
    c.deadline_ms = g->opt.deadline_ms;
    c.search_budget = g->opt.search_budget != 0 ? g->opt.search_budget : P < SMALL_BATCH ? SMALL_BATCH_BUDGET : 0;
    c.split_pieces = g->opt.split_pieces;
    c.sub_searches = g->opt.sub_searches;
    return c;
}

// Map enumerator settings of a set of plans: which passes run, and their limits.
constexpr int32_t EXACT_MIS_DEFAULT_INSTANCES = 2048, EXACT_MIS_MAX_INSTANCES = 4096;
constexpr int32_t EXACT_MIS_BATCH = 64;  // patterns whose maps are materialised at once

void enum_config(const flexis_graph *g, const Plan *plans, int64_t n, EvalConfig &c) {
    c.count_maps = c.exact_mis = false;
    for (int64_t i = 0; i < n; i++) {
        c.count_maps |= plans[i].count_maps != 0;
        c.exact_mis |= plans[i].exact_mis != 0;
    }
    c.maps_cap = g->opt.maps_cap;
    c.frontier_rows = g->opt.frontier_rows;
    c.exact_mis_maps = g->opt.exact_mis_maps > 0 ? std::min(g->opt.exact_mis_maps, EXACT_MIS_MAX_INSTANCES)
                                                 : EXACT_MIS_DEFAULT_INSTANCES;
    c.exact_mis_maps_buffer = std::min(65536, 32 * c.exact_mis_maps);
    c.exact_mis_nodes = g->opt.exact_mis_nodes;
}

// Measured autotuner of the per-round search budget (how far a root search runs before it is
// suspended, resumed or split): on the first batch of a size bucket (power of two of the pattern
// count, >= TUNE_MIN) a slice of the batch is evaluated under each candidate budget, the fastest
// (device time) is kept for the graph and used for the rest of that batch and every later batch
// of the bucket.  All budgets give the same results, so the slice's results are kept as well.
constexpr int32_t TUNE_MIN = 4096;
constexpr int32_t TUNE_CANDIDATES[3] = {1024, 4096, 16384};

int tune_bucket(int64_t P) {
    int b = 0;
    while ((1ll << (b + 1)) <= P) b++;
    return b;
}

// Evaluate plans [lo, lo + cnt) with the autotuner's budget for the bucket (tuning it first if
// the bucket is new).  Returns the results into out + lo.
int eval_chunk(flexis_graph *g, std::vector<Plan> &plans, int64_t lo, int32_t cnt, flexis_support_result *out,
               flexis_stats &total) {
    EvalConfig c2 = config_for(g, cnt);
    enum_config(g, plans.data() + lo, cnt, c2);
    const bool tunable = g->opt.autotune >= 0 && g->opt.search_budget == 0 && cnt >= TUNE_MIN && !c2.exact_mis;
    int64_t done = 0;
    if (tunable) {
        const int bucket = tune_bucket(cnt);
        auto it = g->tuned_budget.find(bucket);
        if (it == g->tuned_budget.end()) {
            const int32_t slice = std::max<int32_t>(512, std::min<int32_t>(cnt / 8, 8192));
            float best_ms = 0.f;
            int32_t best = 0;
            for (int32_t cand : TUNE_CANDIDATES) {
                EvalConfig c3 = config_for(g, slice);
                enum_config(g, plans.data() + lo, slice, c3);
                c3.search_budget = cand;
                c3.w_min = c2.w_min;
                c3.w_max = c2.w_max;
                flexis_stats st{};
                int rc = dev_eval_host(g->dg, plans.data() + lo, slice, out + lo, c3, &st);
                if (rc) return rc;
                st.patterns = slice;
                st.autotune_probes = 1;
                add_stats(total, st);
                if (best == 0 || st.total_ms < best_ms) {
                    best_ms = st.total_ms;
                    best = cand;
                }
            }
            it = g->tuned_budget.emplace(bucket, best).first;
            done = slice;  // every candidate gave these results
        }
        c2.search_budget = it->second;
    }
    if (done < cnt) {
        flexis_stats st{};
        int rc = dev_eval_host(g->dg, plans.data() + lo + done, (int32_t)(cnt - done), out + lo + done, c2, &st);
        if (rc) return rc;
        st.patterns = cnt - done;
        st.batches = 1;
        st.search_budget = c2.search_budget ? c2.search_budget : 4096;
        add_stats(total, st);
    }
    return FLEXIS_OK;
}

// Memory-admitted batches: the device workspace of one batch (used bitmaps, windows, items) is
// bounded by a share of the free device memory; larger candidate sets run as several batches.
int eval_plans(flexis_graph *g, std::vector<Plan> &plans, flexis_support_result *out) {
    const int64_t P = (int64_t)plans.size();
    EvalConfig cfg = config_for(g, (int32_t)std::min<int64_t>(P, INT32_MAX));
    enum_config(g, plans.data(), P, cfg);
    int64_t per = 1, fr = 0;
    dev_pattern_bytes(g->dg, cfg.w_max, cfg.record_selected, &per);
    dev_free_bytes(g->dg, &fr);
    const int64_t budget = std::max<int64_t>(fr / 3, 256ll << 20);
    int64_t chunk = std::max<int64_t>(1, std::min<int64_t>({P, budget / std::max<int64_t>(per, 1), 1 << 22}));
    // the exact MIS materialises every map of its patterns: a few patterns at a time
    if (cfg.exact_mis) chunk = std::min<int64_t>(chunk, EXACT_MIS_BATCH);
    flexis_stats total{};
    for (int64_t lo = 0; lo < P; lo += chunk) {
        const int32_t cnt = (int32_t)std::min(chunk, P - lo);
        int rc = eval_chunk(g, plans, lo, cnt, out, total);
        if (rc) return rc;
    }
    g->last = total;
    return FLEXIS_OK;
}

// A caller's pattern in the form the graph holds: on an edge-labelled graph, each pattern edge
// (a, b) with label l becomes a vertex of label edge_label_base + l joined to a and b (the
// extended pattern of Sec. 2.3.5).  `buf` keeps the extended arrays alive.
struct PatBuf {
    std::vector<int32_t> labels, edges;
};

int user_pattern(const flexis_graph *g, const flexis_pattern &in, PatBuf &buf, flexis_pattern &out) {
    out = in;
    if (g->edge_label_base < 0) {
        if (in.edge_labels) return FLEXIS_E_INVALID;  // edge labels on a graph without them
        return FLEXIS_OK;
    }
    if (!in.edge_labels || in.n < 1 || in.m < 1 || !in.labels || !in.edges || in.n + in.m > MAXN)
        return FLEXIS_E_INVALID;
    buf.labels.assign(in.labels, in.labels + in.n);
    buf.edges.clear();
    std::vector<std::pair<int32_t, int32_t>> seen;
    for (int e = 0; e < in.m; e++) {
        int32_t a = in.edges[2 * e], b = in.edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= in.n || b >= in.n || a == b || in.edge_labels[e] < 0) return FLEXIS_E_INVALID;
        const auto key = std::make_pair(std::min(a, b), std::max(a, b));
        if (std::find(seen.begin(), seen.end(), key) != seen.end()) return FLEXIS_E_INVALID;
        seen.push_back(key);
        const int32_t w = in.n + e;
        buf.labels.push_back(g->edge_label_base + in.edge_labels[e]);
        buf.edges.insert(buf.edges.end(), {a, w, w, b});
    }
    out.n = in.n + in.m;
    out.m = 2 * in.m;
    out.labels = buf.labels.data();
    out.edges = buf.edges.data();
    out.edge_labels = nullptr;
    return FLEXIS_OK;
}

// compile_plan on the graph's form of a caller's pattern (an invalid one gives an error plan)
int compile_user(const flexis_graph *g, const flexis_pattern &pat, int64_t sigma, int64_t num, int64_t den,
                 int mode, Plan &P) {
    PatBuf buf;
    flexis_pattern q;
    const int rc = user_pattern(g, pat, buf, q);
    if (rc) {
        memset(&P, 0, sizeof P);
        P.status = rc;
        P.n = pat.n;
        return rc;
    }
    return compile_plan(g->hg, q, sigma, num, den, mode, P);
}

void pattern_of_code(const flexis_graph *g, const Code &c, std::vector<int32_t> &labels,
                     std::vector<int32_t> &edges) {
    Pat p = pat_of_code(c);
    labels.resize((size_t)p.n);
    edges.clear();
    for (int i = 0; i < p.n; i++) {
        labels[(size_t)i] = g->hg.label_of_rank[(size_t)p.lab[i]];
        for (int j = i + 1; j < p.n; j++)
            if (p.adj[i] >> j & 1) {
                edges.push_back(i);
                edges.push_back(j);
            }
    }
}

}  // namespace

extern "C" {

const char *flexis_status_string(int status) {
    switch (status) {
        case FLEXIS_OK: return "ok";
        case FLEXIS_E_INVALID: return "invalid argument";
        case FLEXIS_E_NOMEM: return "out of memory";
        case FLEXIS_E_CUDA: return "CUDA error";
        case FLEXIS_E_TIMEOUT: return "timeout";
        case FLEXIS_E_CANCELLED: return "cancelled";
        case FLEXIS_E_UNSUPPORTED: return "unsupported graph layout";
        case FLEXIS_E_BUSY: return "busy";
        default: return "unknown status";
    }
}

int flexis_lambda_quantize(double lambda, int64_t *num_out) {
    int64_t num;
    if (!num_out || !lambda_to_q(lambda, &num)) return FLEXIS_E_INVALID;
    *num_out = num;
    return FLEXIS_OK;
}

void flexis_default_options(flexis_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof *opt);
    opt->seed = DEFAULT_SEED;
    opt->device = 0;
}

int flexis_load_graph(int64_t n_vertices, const int32_t *labels, int64_t n_edges,
                      const int32_t *src, const int32_t *dst, const flexis_options *opt,
                      flexis_graph **out) {
    if (!out) return FLEXIS_E_INVALID;
    std::unique_ptr<flexis_graph> g(new (std::nothrow) flexis_graph());
    if (!g) return FLEXIS_E_NOMEM;
    if (opt) g->opt = *opt; else flexis_default_options(&g->opt);
    int rc;
    // the device build sorts 2 x n_edges arcs with 32-bit positions; a larger edge list (and a
    // directed graph) is built on the host
    if (!g->opt.directed && !g->opt.host_build && 2 * (uint64_t)std::max<int64_t>(n_edges, 0) < UINT32_MAX) {
        rc = dev_graph_build(n_vertices, labels, n_edges, src, dst, g->opt.seed, g->opt.root_order == 1,
                             g->opt.device, g->hg, &g->dg);
        if (rc) return rc;
    } else {
        rc = build_host_graph(n_vertices, labels, n_edges, src, dst, g->opt.seed, g->opt.root_order == 1, g->hg,
                              g->opt.directed ? 1 : 0);
        if (rc) return rc;
        rc = dev_graph_create(g->hg, g->opt.device, &g->dg);
        if (rc) return rc;
        // the layout lives on the device; the host keeps the label tables and counts
        std::vector<VRec>().swap(g->hg.vrec);
        std::vector<uint32_t>().swap(g->hg.runs);
        std::vector<int32_t>().swap(g->hg.adj);
        std::vector<int32_t>().swap(g->hg.lab_vtx);
    }
    g->n_input_vertices = n_vertices;
    g->input_self_loops = g->hg.self_loops;
    g->input_duplicates = g->hg.duplicates;
    *out = g.release();
    return FLEXIS_OK;
}

int flexis_load_graph_edge_labels(int64_t n_vertices, const int32_t *labels, int64_t n_edges,
                                  const int32_t *src, const int32_t *dst, const int32_t *edge_labels,
                                  const flexis_options *opt, flexis_graph **out) {
    if (!out || n_vertices < 0 || n_edges < 0 || (n_vertices > 0 && !labels) ||
        (n_edges > 0 && (!src || !dst || !edge_labels)))
        return FLEXIS_E_INVALID;
    int32_t base = 0;
    for (int64_t v = 0; v < n_vertices; v++) {
        if (labels[v] < 0) return FLEXIS_E_INVALID;
        base = std::max(base, labels[v] + 1);
    }
    // kept edges: no self-loop, first occurrence of each vertex pair (either direction)
    std::vector<std::pair<uint64_t, int64_t>> key((size_t)n_edges);
    int64_t loops = 0;
    for (int64_t e = 0; e < n_edges; e++) {
        if (src[e] < 0 || dst[e] < 0 || src[e] >= n_vertices || dst[e] >= n_vertices || edge_labels[e] < 0)
            return FLEXIS_E_INVALID;
        // repeated edges: the same vertex pair (undirected), the same ordered pair (directed)
        const bool dir = opt && opt->directed;
        const uint64_t a = (uint64_t)(dir ? src[e] : std::min(src[e], dst[e]));
        const uint64_t b = (uint64_t)(dir ? dst[e] : std::max(src[e], dst[e]));
        key[(size_t)e] = {a << 32 | b, e};
    }
    std::sort(key.begin(), key.end());
    std::vector<int64_t> kept;
    for (size_t i = 0; i < key.size(); i++) {
        const int64_t e = key[i].second;
        if (src[e] == dst[e]) { loops++; continue; }
        if (i > 0 && key[i - 1].first == key[i].first) continue;
        kept.push_back(e);
    }
    std::sort(kept.begin(), kept.end());
    const int64_t dups = n_edges - loops - (int64_t)kept.size();
    const int64_t nk = (int64_t)kept.size();
    if (n_vertices + nk >= (int64_t)INT32_MAX) return FLEXIS_E_UNSUPPORTED;
    std::vector<int32_t> lab2((size_t)(n_vertices + nk)), s2((size_t)(2 * nk)), d2((size_t)(2 * nk));
    std::copy(labels, labels + n_vertices, lab2.begin());
    for (int64_t k = 0; k < nk; k++) {
        const int64_t e = kept[(size_t)k];
        const int32_t w = (int32_t)(n_vertices + k);
        lab2[(size_t)(n_vertices + k)] = base + edge_labels[e];
        s2[(size_t)(2 * k)] = src[e];
        d2[(size_t)(2 * k)] = w;
        s2[(size_t)(2 * k + 1)] = w;
        d2[(size_t)(2 * k + 1)] = dst[e];
    }
    int rc = flexis_load_graph(n_vertices + nk, lab2.data(), 2 * nk, s2.data(), d2.data(), opt, out);
    if (rc) return rc;
    (*out)->n_input_vertices = n_vertices;
    (*out)->edge_label_base = base;
    (*out)->input_self_loops = loops;
    (*out)->input_duplicates = dups;
    return FLEXIS_OK;
}

int flexis_graph_layout(const flexis_graph *g, int32_t part, void *out, int64_t capacity, int64_t *bytes) {
    if (!g || !bytes) return FLEXIS_E_INVALID;
    return dev_graph_layout(g->dg, part, out, capacity, bytes);
}

void flexis_free_graph(flexis_graph *g) {
    if (!g) return;
    dev_graph_destroy(g->dg);
    delete g;
}

int flexis_graph_info_get(const flexis_graph *g, flexis_graph_info *out) {
    if (!g || !out) return FLEXIS_E_INVALID;
    memset(out, 0, sizeof *out);
    out->n_vertices = g->hg.nv;
    out->n_arcs = g->hg.n_arcs;
    out->n_self_loops = g->input_self_loops;
    out->n_duplicates = g->input_duplicates;
    out->n_input_vertices = g->n_input_vertices;
    out->edge_label_base = g->edge_label_base;
    out->directed = g->opt.directed ? 1 : 0;
    out->n_labels = g->hg.nl;
    out->max_degree = g->hg.max_degree;
    out->device_bytes = dev_graph_bytes(g->dg);
    dev_graph_load_info(g->dg, &out->upload_bytes, &out->built_on_device);
    int sm = 0, l2 = 0;
    dev_graph_props(g->dg, &sm, &l2);
    out->sm_count = sm;
    out->l2_bytes = l2;
    return FLEXIS_OK;
}

int flexis_support_q(flexis_graph *g, const flexis_pattern *pattern, int64_t sigma,
                     int64_t lambda_num, int64_t lambda_den, int32_t mode,
                     flexis_support_result *out) {
    if (!g || !pattern || !out) return FLEXIS_E_INVALID;
    std::vector<Plan> plans(1);
    int rc = compile_user(g, *pattern, sigma, lambda_num, lambda_den, mode, plans[0]);
    if (rc) return rc;
    flexis_support_result r;
    rc = eval_plans(g, plans, &r);
    if (rc) return rc;
    *out = r;
    return FLEXIS_OK;
}

int flexis_support(flexis_graph *g, const flexis_pattern *pattern, int64_t sigma, double lambda,
                   int32_t mode, flexis_support_result *out) {
    int64_t num;
    if (!lambda_to_q(lambda, &num)) return FLEXIS_E_INVALID;
    return flexis_support_q(g, pattern, sigma, num, LAMBDA_DEN, mode, out);
}

int flexis_compile(flexis_graph *g, const flexis_pattern *patterns, const int64_t *sigma,
                   const int64_t *lambda_num, int64_t lambda_den, int32_t count, int32_t mode,
                   flexis_plan *plans_out) {
    if (!g || count < 0 || (count > 0 && (!patterns || !sigma || !lambda_num || !plans_out)))
        return FLEXIS_E_INVALID;
    for (int32_t i = 0; i < count; i++) {
        Plan P;
        compile_user(g, patterns[i], sigma[i], lambda_num[i], lambda_den, mode, P);
        memset(&plans_out[i], 0, sizeof(flexis_plan));
        memcpy(&plans_out[i], &P, sizeof P);
    }
    return FLEXIS_OK;
}

int flexis_support_batch(flexis_graph *g, const flexis_pattern *patterns, const int64_t *sigma,
                         const double *lambda, int32_t count, int32_t mode,
                         flexis_support_result *out) {
    if (!g || count < 0 || (count > 0 && (!patterns || !sigma || !lambda || !out)))
        return FLEXIS_E_INVALID;
    if (count == 0) return FLEXIS_OK;
    std::vector<Plan> plans((size_t)count);
    int T = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (count < 256) T = 1;
    std::vector<std::thread> th;
    auto work = [&](int t) {
        for (int32_t i = t; i < count; i += T) {
            int64_t num = 0;
            if (!lambda_to_q(lambda[i], &num)) {
                memset(&plans[(size_t)i], 0, sizeof(Plan));
                plans[(size_t)i].status = FLEXIS_E_INVALID;
                plans[(size_t)i].n = patterns[i].n;
                continue;
            }
            compile_user(g, patterns[i], sigma[i], num, LAMBDA_DEN, mode, plans[(size_t)i]);
        }
    };
    for (int t = 1; t < T; t++) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();
    return eval_plans(g, plans, out);
}

int flexis_support_plans_device(flexis_graph *g, const flexis_plan *d_plans, int32_t count,
                                flexis_support_result *d_results, void *stream) {
    if (!g || count < 0 || (count > 0 && (!d_plans || !d_results))) return FLEXIS_E_INVALID;
    EvalConfig cfg = config_for(g, count);
    cudaStream_t s = stream ? (cudaStream_t)stream : dev_graph_stream(g->dg);
    if (count > 0) {
        // the plans' mode flags decide which enumerator passes run: read them back (1 KB each)
        std::vector<Plan> h((size_t)count);
        if (cudaMemcpyAsync(h.data(), d_plans, sizeof(Plan) * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return FLEXIS_E_CUDA;
        enum_config(g, h.data(), count, cfg);
    }
    return dev_eval(g->dg, reinterpret_cast<const Plan *>(d_plans), count, d_results, s, cfg, &g->last);
}

int flexis_last_stats(const flexis_graph *g, flexis_stats *out) {
    if (!g || !out) return FLEXIS_E_INVALID;
    *out = g->last;
    return FLEXIS_OK;
}

void *flexis_graph_stream(const flexis_graph *g) { return g ? (void *)dev_graph_stream(g->dg) : nullptr; }

int flexis_support_noalloc(flexis_graph *g, const flexis_plan *plan, flexis_support_result *out,
                           void *stream) {
    if (!g || !plan || !out) return FLEXIS_E_INVALID;
    return dev_support_noalloc(g->dg, reinterpret_cast<const Plan *>(plan), out, (cudaStream_t)stream,
                               g->opt.deadline_ms);
}

int flexis_overlap_graph(flexis_graph *g, const flexis_pattern *pattern, int32_t *instances_out,
                         int64_t cap_instances, int64_t *n_instances, int32_t *edges_out, int64_t cap_edges,
                         int64_t *n_edges) {
    if (!g || !pattern || !n_instances || !n_edges || cap_instances < 0 || cap_edges < 0 ||
        (cap_instances > 0 && !instances_out) || (cap_edges > 0 && !edges_out))
        return FLEXIS_E_INVALID;
    std::vector<Plan> plans(1);
    int rc = compile_user(g, *pattern, 1, 0, 1,
                          FLEXIS_MODE_FULL | FLEXIS_MODE_NO_MNI | FLEXIS_MODE_NO_MIS | FLEXIS_MODE_EXACT_MIS, plans[0]);
    if (rc) return rc;
    flexis_support_result r;
    if ((rc = eval_plans(g, plans, &r))) return rc;
    if (plans[0].flags & FLEXIS_FLAG_ABSENT_LABEL) {
        *n_instances = 0;
        *n_edges = 0;
        return FLEXIS_OK;
    }
    return dev_overlap_read(g->dg, 0, instances_out, cap_instances, n_instances, edges_out, cap_edges, n_edges);
}

int flexis_selected_maps(const flexis_graph *g, int32_t i, int32_t *maps_out, int64_t cap,
                         int64_t *n_out) {
    if (!g || !maps_out || !n_out || cap < 0) return FLEXIS_E_INVALID;
    return dev_selected(g->dg, i, maps_out, cap, n_out);
}

int flexis_mine(flexis_graph *g, int64_t sigma, double lambda, int32_t max_edges,
                flexis_pattern_set **out) {
    int64_t num;
    if (!g || !out || sigma < 1 || max_edges < 1 || !lambda_to_q(lambda, &num)) return FLEXIS_E_INVALID;
    // candidate generation (Algorithms 2-4) is implemented for undirected patterns
    if (g->hg.directed) return FLEXIS_E_UNSUPPORTED;
    std::unique_ptr<flexis_pattern_set> S(new flexis_pattern_set());
    S->label_of_rank = g->hg.label_of_rank;
    // level 2: edges(G), one candidate per label pair on a data edge
    std::vector<Code> C;
    for (auto &pr : g->hg.label_pairs) {
        Code c;
        c.n = 2;
        c.lab[0] = pr.first;
        c.lab[1] = pr.second;
        c.bits = 0;
        C.push_back(c);
    }
    std::sort(C.begin(), C.end());
    const int threads = host_threads();
    flexis_stats total{};
    for (int k = 2; k <= max_edges + 1 && k <= FLEXIS_MAX_PATTERN && !C.empty(); k++) {
        S->cand[k] = (int64_t)C.size();
        std::vector<Plan> plans(C.size());
        auto t0 = Clock::now();
        // candidates are canonical codes over label ranks already; the metric step of
        // Algorithm 1 needs the mIS decision only (Sec. 3.2.2)
        parallel_chunks((int64_t)C.size(), threads, [&](int64_t lo, int64_t hi) {
            for (int64_t i = lo; i < hi; i++) {
                compile_code(g->hg, C[(size_t)i], sigma, num, LAMBDA_DEN,
                             FLEXIS_MODE_EARLY | FLEXIS_MODE_NO_MNI, plans[(size_t)i]);
                plans[(size_t)i].decide_only = 1;
            }
        });
        total.host_compile_ms += ms_since(t0);
        std::vector<flexis_support_result> res(C.size());
        int rc = eval_plans(g, plans, res.data());
        if (rc) return rc;
        add_stats(total, g->last);
        for (size_t i = 0; i < C.size(); i++)
            if (res[i].status == FLEXIS_E_TIMEOUT) {
                g->last = total;
                return FLEXIS_E_TIMEOUT;  // a level with undecided patterns has no frequent set
            }
        std::vector<Code> F;
        for (size_t i = 0; i < C.size(); i++)
            if (res[i].status == FLEXIS_OK && res[i].frequent) {
                // a frequent pattern has mIS >= c, hence MNI >= c: its capped MNI is c
                res[i].mni = res[i].cap;
                res[i].flags = (res[i].flags & ~FLEXIS_FLAG_MNI_SKIPPED) | FLEXIS_FLAG_MNI_FROM_MIS;
                F.push_back(C[i]);
                S->items.push_back({C[i], res[i]});
            }
        S->freq[k] = (int64_t)F.size();
        C.clear();
        t0 = Clock::now();
        if (k + 1 <= max_edges + 1 && k + 1 <= FLEXIS_MAX_PATTERN) generate_candidates(F, max_edges, C, threads);
        total.host_gen_ms += ms_since(t0);
    }
    g->last = total;
    *out = S.release();
    return FLEXIS_OK;
}

int64_t flexis_pattern_set_count(const flexis_pattern_set *s) { return s ? (int64_t)s->items.size() : 0; }

int flexis_pattern_set_get(const flexis_pattern_set *s, int64_t i, int32_t *n, int32_t *labels,
                           int32_t *m, int32_t *edges, int32_t *code_labels, uint32_t *code_bits,
                           flexis_support_result *result) {
    if (!s || i < 0 || i >= (int64_t)s->items.size()) return FLEXIS_E_INVALID;
    const auto &e = s->items[(size_t)i];
    Pat p = pat_of_code(e.code);
    if (n) *n = p.n;
    int mm = 0;
    for (int a = 0; a < p.n; a++) {
        if (labels) labels[a] = s->label_of_rank[(size_t)p.lab[a]];
        if (code_labels) code_labels[a] = e.code.lab[a];
        for (int b = a + 1; b < p.n; b++)
            if (p.adj[a] >> b & 1) {
                if (edges) { edges[2 * mm] = a; edges[2 * mm + 1] = b; }
                mm++;
            }
    }
    if (m) *m = mm;
    if (code_bits) *code_bits = e.code.bits;
    if (result) *result = e.res;
    return FLEXIS_OK;
}

int64_t flexis_pattern_set_read(const flexis_pattern_set *s, int64_t first, int64_t count,
                                int32_t *n_out, int32_t *code_labels, uint32_t *code_bits,
                                int32_t *labels_out, flexis_support_result *results) {
    if (!s || first < 0 || count < 0 || (count > 0 && (!n_out || !code_labels || !code_bits)))
        return FLEXIS_E_INVALID;
    const int64_t end = std::min<int64_t>((int64_t)s->items.size(), first + count);
    for (int64_t i = first; i < end; i++) {
        const auto &e = s->items[(size_t)i];
        const int64_t k = i - first;
        n_out[k] = e.code.n;
        for (int j = 0; j < MAXN; j++) {
            const int32_t r = j < e.code.n ? e.code.lab[j] : 0;
            code_labels[8 * k + j] = r;
            if (labels_out) labels_out[8 * k + j] = j < e.code.n ? s->label_of_rank[(size_t)r] : -1;
        }
        code_bits[k] = e.code.bits;
        if (results) results[k] = e.res;
    }
    return std::max<int64_t>(0, end - first);
}

int flexis_pattern_set_levels(const flexis_pattern_set *s, int64_t *candidates, int64_t *frequent) {
    if (!s) return FLEXIS_E_INVALID;
    for (int k = 0; k <= FLEXIS_MAX_PATTERN; k++) {
        if (candidates) candidates[k] = s->cand[k];
        if (frequent) frequent[k] = s->freq[k];
    }
    return FLEXIS_OK;
}

void flexis_free_pattern_set(flexis_pattern_set *s) { delete s; }

int flexis_canonical_code(const flexis_pattern *pattern, int32_t *labels_out, uint32_t *bits_out,
                          int32_t *perm_out) {
    if (!pattern || !labels_out || !bits_out) return FLEXIS_E_INVALID;
    if (pattern->n < 1 || pattern->n > MAXN || pattern->m < 0 || !pattern->labels || pattern->edge_labels)
        return FLEXIS_E_INVALID;
    Pat p;
    p.n = pattern->n;
    for (int i = 0; i < p.n; i++) p.lab[i] = pattern->labels[i];
    for (int e = 0; e < pattern->m; e++) {
        int a = pattern->edges[2 * e], b = pattern->edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= p.n || b >= p.n || a == b) return FLEXIS_E_INVALID;
        p.adj[a] |= (uint8_t)(1 << b);
        p.adj[b] |= (uint8_t)(1 << a);
    }
    int perm[MAXN];
    Code c = canonical(p, perm);
    for (int i = 0; i < p.n; i++) {
        labels_out[i] = c.lab[i];
        if (perm_out) perm_out[i] = perm[i];
    }
    *bits_out = c.bits;
    return FLEXIS_OK;
}

int64_t flexis_generate_candidates(const flexis_pattern *frequent, int32_t count,
                                   int32_t max_edges, int32_t *n_out, int32_t *labels_out,
                                   uint32_t *bits_out, int64_t cap) {
    if (count < 0 || (count > 0 && !frequent)) return FLEXIS_E_INVALID;
    std::vector<Code> F;
    for (int32_t i = 0; i < count; i++) {
        int32_t lab[MAXN];
        uint32_t bits;
        if (flexis_canonical_code(&frequent[i], lab, &bits, nullptr)) return FLEXIS_E_INVALID;
        Code c;
        c.n = frequent[i].n;
        for (int j = 0; j < c.n; j++) c.lab[j] = lab[j];
        c.bits = bits;
        F.push_back(c);
    }
    std::sort(F.begin(), F.end());
    F.erase(std::unique(F.begin(), F.end()), F.end());
    std::vector<Code> C;
    int threads = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    generate_candidates(F, max_edges, C, threads);
    int64_t n = (int64_t)C.size();
    if (n > cap) return -n;
    for (int64_t i = 0; i < n; i++) {
        n_out[i] = C[(size_t)i].n;
        for (int j = 0; j < MAXN; j++) labels_out[8 * i + j] = j < C[(size_t)i].n ? C[(size_t)i].lab[j] : 0;
        bits_out[i] = C[(size_t)i].bits;
    }
    return n;
}


// ------------------------------------------------------------------ serving
}  // extern "C"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>

struct flexis_server {
    using clock = std::chrono::steady_clock;
    struct Req {
        int64_t id;
        Plan plan;
        clock::time_point t0;
    };
    struct Done {
        int64_t id;
        flexis_support_result res;
        double lat_us;
    };
    flexis_graph *g = nullptr;
    ServeSession *sess = nullptr;
    int32_t slots = 0;
    int32_t deadline_ms = 0;  // per request, from submission; 0 = none
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    int err = FLEXIS_OK;
    std::deque<Req> pending;
    size_t max_pending = 1u << 20;
    std::deque<Done> done;

    void fail(int rc) {
        std::lock_guard<std::mutex> lk(mu);
        err = rc;
        stop = true;
    }

    void loop() {
        std::vector<Req> slot_req((size_t)slots);
        std::vector<char> live((size_t)slots, 0);
        std::vector<int32_t> phase((size_t)slots, 0), admit, cancel;
        std::vector<Plan> aplans;
        std::vector<flexis_support_result> res((size_t)slots);
        int busy = 0;
        for (;;) {
            admit.clear();
            aplans.clear();
            {
                std::unique_lock<std::mutex> lk(mu);
                if (!stop && busy == 0 && pending.empty())
                    cv.wait(lk, [&] { return stop || !pending.empty(); });
                if (stop) break;
                // admission: a free slot is the unit of device memory (used bitmap + window)
                for (int32_t i = 0; i < slots && !pending.empty(); i++) {
                    if (live[(size_t)i]) continue;
                    slot_req[(size_t)i] = pending.front();
                    pending.pop_front();
                    live[(size_t)i] = 1;
                    admit.push_back(i);
                    aplans.push_back(slot_req[(size_t)i].plan);
                    busy++;
                }
            }
            int32_t ng = 0;
            int rc = serve_step(sess, admit.data(), aplans.data(), (int32_t)admit.size(), phase.data(),
                                res.data(), &ng);
            if (rc) { fail(rc); break; }
            auto now = clock::now();
            // requests past their deadline stop before the next step, which reports them
            cancel.clear();
            if (deadline_ms > 0) {
                for (int32_t i = 0; i < slots; i++) {
                    if (!live[(size_t)i] || phase[(size_t)i] == 3) continue;
                    if (std::chrono::duration<double, std::milli>(now - slot_req[(size_t)i].t0).count() > deadline_ms)
                        cancel.push_back(i);
                }
            }
            if (!cancel.empty() && (rc = serve_cancel(sess, cancel.data(), (int32_t)cancel.size())) != 0) {
                fail(rc);
                break;
            }
            std::lock_guard<std::mutex> lk(mu);
            for (int32_t i = 0; i < slots; i++) {
                if (!live[(size_t)i] || phase[(size_t)i] != 3) continue;
                const double us = std::chrono::duration<double, std::micro>(now - slot_req[(size_t)i].t0).count();
                done.push_back(Done{slot_req[(size_t)i].id, res[(size_t)i], us});
                live[(size_t)i] = 0;
                busy--;
            }
        }
    }
};

extern "C" {

int flexis_serve_start(flexis_graph *g, int32_t slots, flexis_server **out) {
    if (!g || !out) return FLEXIS_E_INVALID;
    if (slots <= 0) {
        // admission by memory: a quarter of the free device memory, in slot units
        size_t fr = 0, tot = 0;
        cudaSetDevice(dev_graph_device(g->dg));
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return FLEXIS_E_CUDA;
        int64_t per = 1;
        serve_slot_bytes(g->dg, g->opt.window_max, &per);
        slots = (int32_t)std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t)(fr / 4) / std::max<int64_t>(per, 1)));
    }
    std::unique_ptr<flexis_server> s(new flexis_server());
    s->g = g;
    s->slots = slots;
    s->deadline_ms = g->opt.deadline_ms;
    int rc = serve_create(g->dg, slots, g->opt.window_min, g->opt.window_max, g->opt.search_budget, &s->sess);
    if (rc) return rc;
    flexis_server *raw = s.get();
    s->th = std::thread([raw] { raw->loop(); });
    *out = s.release();
    return FLEXIS_OK;
}

int flexis_serve_submit(flexis_server *s, int64_t request_id, const flexis_pattern *pattern,
                        int64_t sigma, double lambda, int32_t mode) {
    if (!s || !pattern) return FLEXIS_E_INVALID;
    int64_t num;
    if (!lambda_to_q(lambda, &num)) return FLEXIS_E_INVALID;
    flexis_server::Req r;
    r.id = request_id;
    r.t0 = flexis_server::clock::now();
    int rc = compile_user(s->g, *pattern, sigma, num, LAMBDA_DEN, mode, r.plan);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->err) return s->err;
        if (s->stop) return FLEXIS_E_CANCELLED;
        if (s->pending.size() >= s->max_pending) return FLEXIS_E_BUSY;
        s->pending.push_back(r);
    }
    s->cv.notify_all();
    return FLEXIS_OK;
}

int flexis_serve_poll(flexis_server *s, int64_t *ids, flexis_support_result *results,
                      double *latency_us, int32_t max, int32_t *n_out) {
    if (!s || !n_out || max < 0 || (max > 0 && (!ids || !results))) return FLEXIS_E_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    int32_t k = 0;
    while (k < max && !s->done.empty()) {
        auto &d = s->done.front();
        ids[k] = d.id;
        results[k] = d.res;
        if (latency_us) latency_us[k] = d.lat_us;
        s->done.pop_front();
        k++;
    }
    *n_out = k;
    return s->err;
}

int flexis_serve_stop(flexis_server *s) {
    if (!s) return FLEXIS_E_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    int err = s->err;
    serve_destroy(s->sess);
    delete s;
    return err;
}

}  // extern "C"
