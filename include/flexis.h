/*
 * flexis.h -- C ABI of the GB300 support-evaluation library for FLEXIS frequent subgraph mining
 * (arXiv 2404.01585).
 *
 * The library keeps one vertex-labelled data graph resident on one GPU and evaluates the
 * support of candidate patterns in it: the greedy maximal-independent-set count (mIS) of the
 * pattern's maps (Sec. 2.4.3; matcher of Sec. 3.2.2), the minimum-image count (MNI, Sec. 2.4.4)
 * and the frequent decision against the lambda-slider threshold tau (Eq. tau, Sec. 3.1.1).  On
 * top it runs the level-wise mining loop (Algorithm 1) with candidate generation by merging
 * (Algorithms 2-4, Sec. 3.2.1) and a request-serving loop.
 *
 * Conventions (every entry point):
 *   - Return value: FLEXIS_OK (0) or a negative FLEXIS_E_* code; outputs are written only on OK.
 *     flexis_status_string() names a code.  Errors are also reported per pattern in the
 *     `status` field of results.
 *   - Ownership: the caller owns every input array and may free it once the call returns (the
 *     library copies what it keeps).  Handles (flexis_graph, flexis_pattern_set, flexis_server)
 *     are owned by the library and released with the matching flexis_free_* / _stop call.
 *   - Threading: a flexis_graph is thread-compatible, not thread-safe: calls on one handle must
 *     not overlap.  Different handles are independent.  A server owns its own host thread.
 *   - Pointers are host pointers unless the parameter name starts with `d_` (device pointer on
 *     the graph's GPU).
 *   - Exactness: every count is an integer computed exactly; results do not depend on batch
 *     composition, launch shape or the order in which requests arrive.
 *
 * Semantics fixed by this library where the paper leaves a choice open:
 *   - Labels: the labels present in the data graph are ranked by ascending frequency (ties by
 *     id); patterns are canonicalised over ranks.  A pattern label absent from the graph gives
 *     mis = mni = 0 and frequent = 0.
 *   - Which maximal independent set (the paper allows any, Sec. 2.4.3): maps are taken in the
 *     order (H(seed, root), root, lexicographic tuple in matching order), root = image of
 *     canonical vertex 0, H = one SplitMix64 step from state seed XOR root.  Per root the first
 *     map avoiding used vertices is selected and the root's search stops (Sec. 3.2.2, change 1);
 *     used vertices are shared across roots (Sec. 3.2.2, change 2).  options.root_order = 1
 *     drops H: roots are then visited by vertex id.
 *   - tau = floor(sigma * ((n-1) * p + q) / (n * q)) exactly, lambda = p / q, q = 10^6 and
 *     p = llround(lambda * 10^6) for the double-valued entry points.
 *   - Frequent <=> mIS >= max(tau, 1).
 */
#ifndef FLEXIS_H
#define FLEXIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define FLEXIS_OK 0
#define FLEXIS_E_INVALID (-1)     /* bad argument: out-of-range id, disconnected pattern, n<2 or
                                     n>8, lambda outside [0,1] or NaN, sigma < 1, null pointer */
#define FLEXIS_E_NOMEM (-2)       /* a host or device allocation failed */
#define FLEXIS_E_CUDA (-3)        /* a CUDA runtime call failed (no device, launch error) */
#define FLEXIS_E_TIMEOUT (-4)     /* a bounded wait gave up, or a pattern / request / mining run
                                     passed options.deadline_ms before its decision */
#define FLEXIS_E_CANCELLED (-5)   /* a served request was cancelled / server stopped */
#define FLEXIS_E_UNSUPPORTED (-6) /* graph beyond the layout limits (see flexis_load_graph) */
#define FLEXIS_E_BUSY (-7)        /* serving queue full; retry later */

/* ------------------------------------------------------------------ modes */
#define FLEXIS_MODE_FULL 0  /* exact mIS and exact MNI */
#define FLEXIS_MODE_EARLY 1 /* stop at c = max(tau,1) (Sec. 3.1.1): mis = min(mIS, c),
                               mni = min(MNI, c); the frequent decision is unchanged */
#define FLEXIS_MODE_NO_MNI 4 /* or-ed into a mode: skip the MNI count (mni = -1).  The paper's
                                metric step (Sec. 3.2.2) computes the mIS only; mining uses
                                FLEXIS_MODE_EARLY | FLEXIS_MODE_NO_MNI */
#define FLEXIS_MODE_COUNT_MAPS 8 /* or-ed into a mode: also count the set of maps M (Sec. 2.4) into
                                    n_maps, by a level-by-level enumeration of all maps (not only
                                    the greedy's first map per root); saturates at
                                    options.maps_cap (FLEXIS_FLAG_MAPS_SATURATED) */
#define FLEXIS_MODE_NO_MIS 16 /* or-ed into a mode: skip the greedy mIS phase (mis = -1,
                                 frequent = 0, FLEXIS_FLAG_MIS_SKIPPED).  With
                                 FLEXIS_MODE_COUNT_MAPS | FLEXIS_MODE_FULL this is the count-only
                                 mode: |M| and the exact MNI (Sec. 2.4.4) without the greedy */
#define FLEXIS_MODE_EXACT_MIS 32 /* or-ed into a mode: also compute the maximum independent set of
                                    the overlap graph (MIS, Sec. 2.4.2) into mis_exact, for small
                                    overlap graphs: all maps are materialised, reduced to distinct
                                    instances (image vertex sets), conflict edges are built from a
                                    vertex -> instance index, and a branch-and-bound search runs on
                                    the device.  Beyond options.exact_mis_maps instances or
                                    options.exact_mis_nodes search nodes the result is a lower
                                    bound flagged FLEXIS_FLAG_EXACT_MIS_SATURATED */

/* result flags */
#define FLEXIS_FLAG_ABSENT_LABEL 1u /* a pattern label does not occur in the data graph */
#define FLEXIS_FLAG_MNI_FROM_MIS 2u /* mni follows from mis (mis reached c, or M is empty) */
#define FLEXIS_FLAG_MNI_SKIPPED 4u  /* FLEXIS_MODE_NO_MNI: mni not computed (-1) */
#define FLEXIS_FLAG_MIS_SATURATED 8u  /* EARLY: mis reached c; the pattern's mIS may be larger */
#define FLEXIS_FLAG_MNI_SATURATED 16u /* EARLY: mni reached c; the pattern's MNI may be larger */
#define FLEXIS_FLAG_MAPS_SATURATED 32u /* n_maps reached options.maps_cap; |M| may be larger */
#define FLEXIS_FLAG_MIS_SKIPPED 64u   /* FLEXIS_MODE_NO_MIS: the greedy phase did not run */
#define FLEXIS_FLAG_EXACT_MIS_SATURATED 128u /* mis_exact is a lower bound (instance or node limit) */

#define FLEXIS_MAX_PATTERN 8 /* largest pattern, in vertices */

typedef struct flexis_graph flexis_graph;
typedef struct flexis_pattern_set flexis_pattern_set;
typedef struct flexis_server flexis_server;

typedef struct {
    uint64_t seed;        /* greedy-order seed (default 0x5EED) */
    int32_t device;       /* CUDA device ordinal (default 0) */
    int32_t window_min;   /* speculation window per pattern: 0 = autotuned */
    int32_t window_max;   /* 0 = autotuned */
    int32_t search_blocks;/* blocks of the search kernel: 0 = autotuned (multiple of the SM count) */
    int32_t record_selected; /* >0: keep up to this many selected maps per pattern (tests) */
    int32_t search_budget;   /* candidate chunks a root search runs per round before it is
                                suspended and resumed in the next round (earlier, after 32 chunks,
                                once nearly all of the search launch is out of work): 0 = default,
                                -1 = never */
    int32_t split_pieces;    /* pieces a suspended search heading its slot is split into per round:
                                0 = default, -1 = never split */
    int32_t sub_searches;    /* saved sub-searches a pattern may hold at once (1..32): 0 = default */
    int32_t timing;          /* 1: CUDA events around every search launch (stats.search_ms) */
    int32_t graphs;          /* 0 = default (the round loop of each level is captured once into a
                                CUDA graph and replayed), -1 = launch kernel by kernel */
    int32_t deadline_ms;     /* > 0: wall-clock limit of one evaluation call (support, batch, each
                                device batch of a mining level) and of one served request (from
                                its submission).  Patterns still undecided when it passes stop
                                between two rounds and report status FLEXIS_E_TIMEOUT, with mis =
                                the maps committed so far (a lower bound of their mIS), mni = -1
                                and frequent = 0 (undecided); flexis_mine then fails with
                                FLEXIS_E_TIMEOUT.  The limit is checked between rounds of the
                                greedy phase, and by the MNI kernel itself (device clock) every
                                few thousand candidate chunks of a search: a pattern whose MNI
                                count is cut reports FLEXIS_E_TIMEOUT with its final mis and
                                frequent and mni = -1.  0 = no limit (default). */
    int32_t root_order;      /* greedy root order (Sec. 3.2.2): 0 = by (H(seed, v), v), the seeded
                                hash order (default); 1 = by vertex id, the order in which the
                                paper's matcher visits the data vertices (seed unused) */
    int32_t directed;        /* 0 = undirected data graph (each edge read both ways, the paper's
                                loader, Sec. 4.1); 1 = directed: (src[e], dst[e]) is one arc and
                                pattern edges are arcs too (the paper's directed matcher, Sec. 2.2) */
    int64_t maps_cap;        /* FLEXIS_MODE_COUNT_MAPS: n_maps saturates here (0 = 2^32) */
    int64_t frontier_rows;   /* rows of one level of the map enumerator's frontier (0 = 2^22);
                                raised to at least the largest vertex degree */
    int64_t exact_mis_nodes; /* FLEXIS_MODE_EXACT_MIS: branch-and-bound nodes per pattern (0 = 2^24) */
    int32_t exact_mis_maps;  /* FLEXIS_MODE_EXACT_MIS: largest number of distinct instances whose
                                overlap graph is searched (0 = 2048, at most 4096) */
    int32_t autotune;        /* 0 = default: the first batch of >= 4096 patterns of each size
                                (power-of-two bucket) times a slice of itself under a few per-round
                                search budgets and keeps the fastest for the graph; -1 = off (the
                                built-in table).  Results never depend on it */
    int32_t host_build;      /* 0 = default: an undirected graph's layout is built on the device
                                from the uploaded edge list (a radix sort of the arcs); 1 = built
                                on the host and uploaded.  Both give the same arrays bit for bit;
                                a directed graph is always built on the host */
    int32_t reserved[4];
} flexis_options;

/* A query pattern: n vertices with labels[n] (label ids of the data graph), m undirected
 * edges edges[2*m] as 0-based vertex pairs.  Repeated edges are allowed and merged; self-loops
 * and disconnected patterns are FLEXIS_E_INVALID.  2 <= n <= 8.
 * edge_labels[m]: labels of the edges, for graphs loaded with flexis_load_graph_edge_labels
 * (required there, and NULL otherwise).  Such a pattern is evaluated in its extended form (each
 * edge subdivided by a vertex carrying the edge's label, Sec. 2.3.5), which must have at most
 * 8 vertices (n + m <= 8) and no repeated edge.                                              */
typedef struct {
    int32_t n;
    int32_t m;
    const int32_t *labels;
    const int32_t *edges;
    const int32_t *edge_labels;
} flexis_pattern;

/* Support of one pattern (all integer). */
typedef struct {
    int32_t status;   /* FLEXIS_OK or an error code for this pattern */
    int32_t n;        /* pattern vertices */
    int64_t sigma;
    int64_t tau;      /* Eq. tau */
    int64_t cap;      /* EARLY: max(tau,1); FULL: -1 */
    int64_t mis;      /* greedy maximal independent set size (capped in EARLY mode) */
    int64_t mni;      /* minimum image count (capped in EARLY mode) */
    int32_t frequent; /* mis >= max(tau, 1) */
    uint32_t flags;   /* FLEXIS_FLAG_* */
    uint64_t n_maps;  /* FLEXIS_MODE_COUNT_MAPS: |M|, the number of maps (Sec. 2.4; automorphic
                         maps counted separately), saturating at options.maps_cap; else 0 */
    int64_t mis_exact;/* FLEXIS_MODE_EXACT_MIS: size of a maximum independent set of the maps
                         (Sec. 2.4.2); else -1 */
    int64_t roots_searched; /* diagnostics below: not part of the result                      */
                            /* root searches run by the greedy phase                          */
    int64_t search_steps;   /* candidate chunks scanned by those searches                     */
    int32_t max_item_steps; /* largest chunk count of one root search                         */
    int32_t rounds;         /* speculation rounds the pattern took part in                    */
} flexis_support_result;

/* Precompiled pattern (host-side pattern compilation: canonical form, automorphism orbits,
 * matching orders, tau).  Plain bytes: may be copied to device memory and passed to
 * flexis_support_plans_device.                                                                 */
typedef struct {
    uint8_t bytes[1024];
} flexis_plan;

typedef struct {
    int64_t n_vertices;
    int64_t n_arcs;           /* directed arcs kept (2 x undirected edges) */
    int64_t n_self_loops;     /* dropped */
    int64_t n_duplicates;     /* dropped (undirected repeats) */
    int32_t n_labels;         /* labels present */
    int32_t max_degree;
    int64_t device_bytes;     /* device memory held by the graph */
    int32_t sm_count;
    int32_t l2_bytes;
    int64_t n_input_vertices; /* vertices the caller passed (before the edge-label extension) */
    int32_t edge_label_base;  /* label id of edge label 0 in the extended graph; -1 without
                                 edge labels */
    int32_t directed;         /* 1 for a directed graph (options.directed) */
    int32_t built_on_device;  /* 1: the layout was built on the device (options.host_build) */
    int64_t upload_bytes;     /* host-to-device bytes of the load: the edge list and vertex ranks
                                 (device build) or the layout arrays (host build) */
} flexis_graph_info;

/* Counters of the last support / batch / mining call on a graph (diagnostics, timing). */
typedef struct {
    int64_t rounds;           /* speculation rounds */
    int64_t search_items;     /* root searches run by the search kernel */
    int64_t mni_items;        /* existence searches run by the MNI kernel */
    int64_t kernel_launches;  /* kernels launched by the call */
    int64_t alg_bytes;        /* algorithmic bytes of the search kernels: the greedy search's
                                 (below) plus the MNI searches' touched bytes (adjacency entries,
                                 label-run entries, vertex records) */
    int64_t alg_bytes_greedy; /* greedy search kernel: 4 * search_scanned + 8 * search_bound +
                                 4 * search_map_words */
    int64_t patterns;         /* patterns evaluated by the call */
    int64_t h2d_bytes;        /* bytes copied host -> device (plans) */
    int64_t d2h_bytes;        /* bytes copied device -> host (results, control words) */
    float search_ms;          /* summed CUDA-event time of the greedy search kernel launches
                                 (measured with options.timing = 1, else 0) */
    float mni_ms;             /* CUDA-event time of the MNI kernel (options.timing = 1) */
    float total_ms;           /* CUDA-event time of the device sections */
    float host_gen_ms;        /* host time in candidate generation (mining) */
    float host_compile_ms;    /* host time in pattern compilation */
    int32_t search_launches;  /* launches of the greedy search kernel */
    int32_t batches;          /* device batches (memory-admitted chunks of the patterns) */
    int32_t graph_launches;   /* replays of the captured round-loop CUDA graph (each runs the
                                 rounds between two host checks); 0 when launched one by one */
    int64_t enum_rows;        /* map enumerator (FLEXIS_MODE_COUNT_MAPS / _EXACT_MIS): partial
                                 maps extended */
    int64_t enum_scanned;     /* ... label-slice entries scanned by those extensions */
    int64_t enum_bytes;       /* ... algorithmic bytes read by them */
    int64_t search_scanned;   /* greedy search kernel: label-slice entries scanned as candidates
                                 (the A of the algorithmic-bytes model) */
    int64_t search_bound;     /* ... partial maps it bound, each counted with its length (level+1):
                                 sum over levels i of (i+1) E_i */
    int64_t search_map_words; /* ... vertex ids of the maps it found and wrote (n per map) */
    int32_t autotune_probes;  /* slice evaluations the autotuner timed in this call */
    int32_t search_budget;    /* per-round search budget of the last batch (tuned or table) */
} flexis_stats;

const char *flexis_status_string(int status);

/* lambda as the exact rational num / FLEXIS_LAMBDA_DEN used by every double-valued entry point
 * (Eq. tau takes lambda in [0, 1]): num = llround(lambda * 10^6), i.e. halves round away from
 * zero.  FLEXIS_E_INVALID for lambda outside [0, 1] or NaN (num_out untouched).  Callers that
 * compile plans with flexis_compile use this to get the same tau as flexis_support.           */
#define FLEXIS_LAMBDA_DEN 1000000
int flexis_lambda_quantize(double lambda, int64_t *num_out);

/* Fill *opt with the defaults. */
void flexis_default_options(flexis_options *opt);

/* Load a data graph (Sec. 2.2: single large vertex-labelled graph; undirected, as the paper's
 * loader, Sec. 4.1).  labels[n_vertices] >= 0; src/dst[n_edges] vertex ids in [0, n_vertices).
 * Self-loops and repeated edges are dropped (counted in flexis_graph_info).  The graph is kept
 * on the device as a CSR with adjacency sorted by (label rank, id), a per-vertex label-run table
 * and a label-partitioned vertex index in greedy-root order.  An undirected graph's layout is
 * built on the device from the uploaded edge list (options.host_build selects the host builder;
 * both give the same arrays); the caller's arrays are only read during the call.
 * Layout limits (FLEXIS_E_UNSUPPORTED beyond them): fewer than 255 distinct labels present,
 * n_vertices < 2^31, directed arcs < 2^32, vertex degree < 2^24.  opt may be NULL.             */
int flexis_load_graph(int64_t n_vertices, const int32_t *labels, int64_t n_edges,
                      const int32_t *src, const int32_t *dst, const flexis_options *opt,
                      flexis_graph **out);

/* Load an edge-labelled data graph (Sec. 2.3.5, extended core graphs): every kept edge (u, v)
 * with label edge_labels[e] >= 0 is replaced by two edges (u, w), (w, v) through a new vertex w
 * whose label is edge_label_base + edge_labels[e], edge_label_base = 1 + the largest vertex
 * label.  The resident graph is that vertex-labelled extended graph (n_vertices + kept edges
 * vertices; flexis_graph_info reports both counts and the base), and every evaluation, mining
 * run and served request works on it: a pattern passes its edge labels in
 * flexis_pattern.edge_labels and is extended the same way, so tau, mis and mni are those of the
 * extended pattern (n + m vertices).  Mined patterns are vertex-labelled patterns of the extended
 * graph.  Self-loops are dropped; of repeated edges between the same two vertices (in either
 * direction) the first one, with its label, is kept.                                          */
int flexis_load_graph_edge_labels(int64_t n_vertices, const int32_t *labels, int64_t n_edges,
                                  const int32_t *src, const int32_t *dst, const int32_t *edge_labels,
                                  const flexis_options *opt, flexis_graph **out);
void flexis_free_graph(flexis_graph *g);
int flexis_graph_info_get(const flexis_graph *g, flexis_graph_info *out);

/* Copy one array of the resident layout to host memory (diagnostics and tests).  part:
 * FLEXIS_LAYOUT_VREC (8 x uint32 per record: adjacency offset, run offset, degree,
 * runs << 8 | rank label, the 64-bit set of neighbour rank labels < 64, 8 zero bytes; one record
 * per vertex, three per vertex for a directed graph: out, in, mutual), FLEXIS_LAYOUT_RUNS
 * (uint32: rank << 24 | slice offset per label run, then 0xFF << 24 | degree, per vertex),
 * FLEXIS_LAYOUT_ADJ (int32 neighbour ids sorted by (rank label, id) per vertex) or
 * FLEXIS_LAYOUT_LAB_VTX (int32 vertex ids grouped by rank label, in greedy-root order).
 * *bytes receives the array's size; out == NULL only queries it; capacity (bytes) below that
 * size is FLEXIS_E_INVALID.  Synchronous.                                                      */
#define FLEXIS_LAYOUT_VREC 0
#define FLEXIS_LAYOUT_RUNS 1
#define FLEXIS_LAYOUT_ADJ 2
#define FLEXIS_LAYOUT_LAB_VTX 3
int flexis_graph_layout(const flexis_graph *g, int32_t part, void *out, int64_t capacity, int64_t *bytes);

/* Support of one pattern (Sec. 2.4, Eq. tau): one plain evaluation, launched and synchronised
 * on its own.  lambda in [0,1]; mode FLEXIS_MODE_EARLY or FLEXIS_MODE_FULL.                    */
int flexis_support(flexis_graph *g, const flexis_pattern *pattern, int64_t sigma, double lambda,
                   int32_t mode, flexis_support_result *out);

/* Same with lambda = lambda_num / lambda_den exactly. */
int flexis_support_q(flexis_graph *g, const flexis_pattern *pattern, int64_t sigma,
                     int64_t lambda_num, int64_t lambda_den, int32_t mode,
                     flexis_support_result *out);

/* Supports of `count` patterns evaluated together (all candidates of a mining level,
 * Algorithm 1 / Algorithm 5 loop): one batched device pass.  sigma[count], lambda[count].
 * Per-pattern errors go to out[i].status; the call fails only on device errors.                */
int flexis_support_batch(flexis_graph *g, const flexis_pattern *patterns, const int64_t *sigma,
                         const double *lambda, int32_t count, int32_t mode,
                         flexis_support_result *out);

/* Host-side pattern compilation into plans (see flexis_plan).  Per-pattern errors are stored
 * in the plan and reported by the evaluation; returns FLEXIS_E_INVALID only for bad arrays.    */
int flexis_compile(flexis_graph *g, const flexis_pattern *patterns, const int64_t *sigma,
                   const int64_t *lambda_num, int64_t lambda_den, int32_t count, int32_t mode,
                   flexis_plan *plans_out);

/* Batched evaluation of plans already resident in device memory; results written to device
 * memory d_results[count].  Runs on `stream` (a cudaStream_t, NULL = the graph's stream) and
 * returns after the results are written (the call synchronises the stream).                    */
int flexis_support_plans_device(flexis_graph *g, const flexis_plan *d_plans, int32_t count,
                                flexis_support_result *d_results, void *stream);

/* Support of one compiled pattern without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc during evaluation -- code that
 * runs under a device-memory budget owned by another framework (whose allocator it must not
 * bypass), or on a latency-critical path where cudaMalloc/cudaFree would implicitly synchronise
 * the device.  All device scratch (control words, pattern state, window buffers, work items,
 * saved searches, used-vertex bitmap) comes from one static device array of 8 MiB that every GPU
 * loading this library holds until the process exits; the call allocates nothing (no cudaMalloc,
 * no cudaFree, no allocating library routine).
 *   plan   : host pointer to one plan from flexis_compile (the caller passes the input)
 *   out    : host pointer, receives the result (same values as flexis_support on that pattern)
 *   stream : cudaStream_t to run on, NULL = the graph's stream; the call synchronises it
 * The graph's options.deadline_ms applies as in flexis_support: a pattern still undecided when it
 * passes stops between two rounds with status FLEXIS_E_TIMEOUT.
 * Limits: one pattern per call, speculation window of 1024 roots, and the used-vertex bitmap
 * (n_vertices / 8 bytes) must fit the array beside about 96 KiB of other scratch, i.e. graphs of
 * up to about 66 million vertices; larger graphs return FLEXIS_E_UNSUPPORTED with the exact limit
 * printed on stderr.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, once per
 * device).  Every call on a device shares the
 * array and it keeps the last call's contents (the call clears what must start at zero): calls
 * whose work overlaps on the GPU -- on different streams or from different threads -- race, so
 * serialise them.                                                                               */
int flexis_support_noalloc(flexis_graph *g, const flexis_plan *plan, flexis_support_result *out,
                           void *stream);

/* Overlap graph of one pattern (Sec. 2.4.1: two maps overlap when they share a data vertex),
 * built on the device as for FLEXIS_MODE_EXACT_MIS: every map is enumerated, maps with the same
 * image vertex set are merged into one instance, a data-vertex -> instance index is built by
 * sorting (vertex, instance) keys, and each vertex's run of instances gives conflict edges.
 *   instances_out : cap_instances rows of 8 ids (an instance's vertices ascending, -1 padded),
 *                   rows in ascending lexicographic order; *n_instances = their number
 *   edges_out     : cap_edges pairs (a, b), a < b, instance indices whose vertex sets meet, in
 *                   ascending order; *n_edges = their number
 * At most cap_* entries are written (the counts are complete).  FLEXIS_E_UNSUPPORTED (with
 * *n_instances = -1) when the pattern has more maps or instances than the limits of
 * FLEXIS_MODE_EXACT_MIS (options.exact_mis_maps).  A label absent from the graph gives 0 / 0. */
int flexis_overlap_graph(flexis_graph *g, const flexis_pattern *pattern, int32_t *instances_out,
                         int64_t cap_instances, int64_t *n_instances, int32_t *edges_out,
                         int64_t cap_edges, int64_t *n_edges);

/* Counters of the last evaluation call on g. */
int flexis_last_stats(const flexis_graph *g, flexis_stats *out);

/* The CUDA stream (a cudaStream_t) on which g's evaluations run, for callers that time them
 * with CUDA events or order their own work after them.  Owned by the graph.                    */
void *flexis_graph_stream(const flexis_graph *g);

/* Selected maps recorded by the last evaluation when opt.record_selected > 0: for pattern i,
 * up to `cap` maps of 8 ids each (canonical-vertex order, in selection order) into maps_out;
 * *n_out gets their number.                                                                    */
int flexis_selected_maps(const flexis_graph *g, int32_t i, int32_t *maps_out, int64_t cap,
                         int64_t *n_out);

/* Mining (Algorithm 1): level 2 = label pairs present on data edges; each level evaluated as
 * one batch in EARLY mode; next candidates by merging (Algorithms 2-4, Sec. 3.2.1) with
 * canonical-code duplicate removal; levels k = 2 .. max_edges+1 vertices, keeping candidates
 * with at most max_edges edges.  The set is sorted by (n, canonical code).                     */
int flexis_mine(flexis_graph *g, int64_t sigma, double lambda, int32_t max_edges,
                flexis_pattern_set **out);
int64_t flexis_pattern_set_count(const flexis_pattern_set *s);
/* i-th frequent pattern in canonical form: *n, labels[8] (label ids), *m, edges[2*28],
 * rank-space canonical code (code_labels[8] ranks, *code_bits), and its support result.        */
int flexis_pattern_set_get(const flexis_pattern_set *s, int64_t i, int32_t *n, int32_t *labels,
                           int32_t *m, int32_t *edges, int32_t *code_labels, uint32_t *code_bits,
                           flexis_support_result *result);
/* Patterns first .. first+count-1 in one call: n_out[count], code_labels[count*8] (label ranks in
 * canonical order), code_bits[count], labels_out[count*8] (label ids, nullable),
 * results[count] (nullable).  Returns the number written (fewer at the end of the set).       */
int64_t flexis_pattern_set_read(const flexis_pattern_set *s, int64_t first, int64_t count,
                                int32_t *n_out, int32_t *code_labels, uint32_t *code_bits,
                                int32_t *labels_out, flexis_support_result *results);
/* per level k (0..8): candidates evaluated and frequent patterns found */
int flexis_pattern_set_levels(const flexis_pattern_set *s, int64_t *candidates, int64_t *frequent);
void flexis_free_pattern_set(flexis_pattern_set *s);

/* Canonical code of a pattern with its labels used as given (the form that replaces Bliss's,
 * Sec. 2.1.5): labels in canonical order, adjacency bits, and perm[p] = input vertex at
 * canonical position p.                                                                        */
int flexis_canonical_code(const flexis_pattern *pattern, int32_t *labels_out, uint32_t *bits_out,
                          int32_t *perm_out);

/* Candidate generation by core-group merging (Algorithms 2-4) on patterns given with labels
 * used as given.  Writes sorted canonical codes (n, labels[8], bits) of the candidates; returns
 * their number, or -(number) if cap is too small.  max_edges <= 0: no edge limit.            */
int64_t flexis_generate_candidates(const flexis_pattern *frequent, int32_t count,
                                   int32_t max_edges, int32_t *n_out, int32_t *labels_out,
                                   uint32_t *bits_out, int64_t cap);

/* ------------------------------------------------------------------ serving
 * A server keeps the graph resident and evaluates support requests as they arrive
 * (continuous batching): requests are admitted into device slots while earlier ones are still
 * being evaluated, and share the device rounds with them.  A slot (used-vertex bitmap, window,
 * state: the device memory one request holds) is the admission unit; slots <= 0 sizes the
 * server from a quarter of the free device memory.  The server's host thread runs rounds of 256
 * candidate chunks per search and request on its own CUDA stream.  The graph's options.deadline_ms, when set, bounds each request from its
 * submission: a request past it is reported with status FLEXIS_E_TIMEOUT (see flexis_options).
 * window_min / window_max / search_budget of the graph's options, when set, replace the
 * server's own defaults (start window 32, at most 2048).                                      */
int flexis_serve_start(flexis_graph *g, int32_t slots, flexis_server **out);
/* Queue a request; copies the pattern.  FLEXIS_E_BUSY if the host queue is full. */
int flexis_serve_submit(flexis_server *s, int64_t request_id, const flexis_pattern *pattern,
                        int64_t sigma, double lambda, int32_t mode);
/* Take up to `max` finished results; ids[i] is the request id of results[i]; latency_us[i] the
 * time from submit to completion (nullable). Non-blocking.                                     */
int flexis_serve_poll(flexis_server *s, int64_t *ids, flexis_support_result *results,
                      double *latency_us, int32_t max, int32_t *n_out);
/* Stop: pending requests finish with FLEXIS_E_CANCELLED.  Frees the server. */
int flexis_serve_stop(flexis_server *s);

#ifdef __cplusplus
}
#endif
#endif /* FLEXIS_H */
