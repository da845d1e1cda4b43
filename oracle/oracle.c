/*
 * FLEXIS support-evaluation ORACLE -- plain, slow, obviously-correct CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this library: only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark do.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only in the seeded input
 * generators (which hold none of the method's arithmetic).
 *
 * Paper: "FLEXIS: FLEXible frequent subgraph mIning using maximal independent Sets",
 * arXiv 2404.01585.  Each function names the passage it follows.  Where the paper leaves a
 * choice open (which maximal independent set, the matching order, the canonical form that
 * replaces Bliss), the oracle follows one fixed reading, written out where it is used:
 *
 *   R1 label ranks   : labels present in the data graph are renumbered by ascending frequency
 *                      (ties by label id); everything below works on ranks.
 *   R2 canonical form: the lexicographic minimum, over all n! vertex orders, of
 *                      (n, rank labels in order, then for j = 1..n-1 and i = 0..j-1 the bit
 *                      "position i is NOT adjacent to position j").
 *   R3 matching order: pi_0 = canonical position 0; pi_{k+1} = the smallest unvisited canonical
 *                      position adjacent to a visited one.
 *   R4 greedy order  : maps sorted by (H(seed, root), root, e[pi_1], ..., e[pi_{n-1}]) with
 *                      root = e[pi_0] and H(s, r) = SplitMix64 step from state s XOR r
 *                      (Steele, Lea, Flood 2014).  The mIS is the sequential greedy independent
 *                      set over M in that order (Sec. 2.4.3 maximal independent set; Sec. 3.2.2
 *                      matcher: one match per root, shared used-vertex bitmap).
 *                      Root-order variant "id" (or_graph_set_root_order): H is dropped, roots
 *                      are visited in vertex-id order, the order in which the paper's own
 *                      matcher walks the data graph's vertices (Sec. 3.2.2).
 *   R5 early mode    : counts are reported as min(count, c) with c = max(tau, 1) (Sec. 3.1.1:
 *                      stop once tau is reached); frequent <=> mIS >= max(tau, 1).
 *
 * Pins (tests/): the paper's running example (Fig. 1, Sec. 2.2, Sec. 2.4.4, Sec. 3.1.1), the
 * Theorem 1 tightness example (Fig. malVisual), brute-force agreement of the two tiers below,
 * Theorem 1 bounds against a brute-force maximum independent set, networkx isomorphism for the
 * canonical code, the candidate-generation figures (Sec. 3.2.1), and for the mining loop
 * (Algorithm 1) a separate level-wise miner written in plain Python over brute-force maps.  No
 * function here is unpinned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 8

/* ------------------------------------------------------------------ tau, Eq. (tau), Sec. 3.1.1
 * tau = floor( sigma * (1 - 1/n) * lambda + sigma / n ), lambda = num / den, evaluated exactly:
 *     = floor( sigma * ((n - 1) * num + den) / (n * den) ).                                     */
int64_t or_tau(int64_t sigma, int64_t lam_num, int64_t lam_den, int32_t n)
{
    __int128 top = (__int128)sigma * ((__int128)(n - 1) * lam_num + lam_den);
    __int128 bot = (__int128)n * lam_den;
    return (int64_t)(top / bot); /* all terms non-negative: truncation == floor */
}

/* ------------------------------------------------------------------ R4 hash */
uint64_t or_hash(uint64_t seed, int64_t r)
{
    uint64_t z = (seed ^ (uint64_t)r) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ data graph (Sec. 2.2)
 * Simple, vertex-labelled; undirected (each edge read both ways, the paper's loader, Sec. 4.1)
 * or directed (each edge one arc src -> dst: the paper states the problem on directed graphs,
 * Sec. 2.2).  Self-loops and repeated edges (arcs) are dropped.                               */
typedef struct {
    int64_t nv;
    int32_t nl;          /* label ids are 0..nl-1 */
    int32_t *rank_of;    /* [nl] rank of a label (R1), -1 if the label has no vertex */
    int32_t *lab;        /* [nv] rank label of each vertex */
    int64_t *off;        /* [nv+1] */
    int32_t *nbr;        /* out-neighbours (all neighbours when undirected), sorted by id */
    int64_t *ioff;       /* directed: [nv+1] */
    int32_t *inbr;       /* directed: in-neighbours, sorted by id */
    int directed;
    uint64_t seed;
    int id_order;        /* 1: roots in vertex-id order (no hash key) */
} or_graph;

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* sorted, repeat-free rows of a list of (row, value) pairs: off[nv+1], nbr */
static void build_rows(int64_t nv, int64_t ne, const int32_t *row, const int32_t *val, const int32_t *skip_a,
                       const int32_t *skip_b, int64_t **off_out, int32_t **nbr_out)
{
    int64_t *deg = calloc(nv + 1, sizeof *deg);
    for (int64_t e = 0; e < ne; e++)
        if (skip_a[e] != skip_b[e]) deg[row[e]]++;
    int64_t *start = malloc((nv + 1) * sizeof *start);
    start[0] = 0;
    for (int64_t v = 0; v < nv; v++) start[v + 1] = start[v] + deg[v];
    int32_t *tmp = malloc((start[nv] > 0 ? start[nv] : 1) * sizeof *tmp);
    int64_t *fill = calloc(nv + 1, sizeof *fill);
    for (int64_t e = 0; e < ne; e++)
        if (skip_a[e] != skip_b[e]) tmp[start[row[e]] + fill[row[e]]++] = val[e];
    int64_t *off = malloc((nv + 1) * sizeof *off);
    int32_t *nbr = malloc((start[nv] > 0 ? start[nv] : 1) * sizeof *nbr);
    int64_t k = 0;
    for (int64_t v = 0; v < nv; v++) {
        off[v] = k;
        int32_t *r = tmp + start[v];
        qsort(r, (size_t)deg[v], sizeof *r, cmp_i32);
        for (int64_t i = 0; i < deg[v]; i++)
            if (i == 0 || r[i] != r[i - 1]) nbr[k++] = r[i];
    }
    off[nv] = k;
    free(deg); free(start); free(tmp); free(fill);
    *off_out = off;
    *nbr_out = nbr;
}

void *or_graph_new2(int64_t nv, const int32_t *labels, int64_t ne, const int32_t *src,
                    const int32_t *dst, uint64_t seed, int directed)
{
    or_graph *g = calloc(1, sizeof *g);
    g->nv = nv;
    g->seed = seed;
    g->directed = directed ? 1 : 0;
    int32_t nl = 0;
    for (int64_t v = 0; v < nv; v++)
        if (labels[v] + 1 > nl) nl = labels[v] + 1;
    g->nl = nl;
    int64_t *cnt = calloc(nl > 0 ? nl : 1, sizeof *cnt);
    for (int64_t v = 0; v < nv; v++) cnt[labels[v]]++;
    g->rank_of = malloc((nl > 0 ? nl : 1) * sizeof *g->rank_of);
    /* R1: rank = number of present labels that come before this one in (count, id) order */
    for (int32_t a = 0; a < nl; a++) {
        if (cnt[a] == 0) { g->rank_of[a] = -1; continue; }
        int32_t r = 0;
        for (int32_t b = 0; b < nl; b++)
            if (cnt[b] > 0 && (cnt[b] < cnt[a] || (cnt[b] == cnt[a] && b < a))) r++;
        g->rank_of[a] = r;
    }
    free(cnt);
    g->lab = malloc((nv > 0 ? nv : 1) * sizeof *g->lab);
    for (int64_t v = 0; v < nv; v++) g->lab[v] = g->rank_of[labels[v]];

    if (g->directed) {
        build_rows(nv, ne, src, dst, src, dst, &g->off, &g->nbr);    /* out-neighbours */
        build_rows(nv, ne, dst, src, src, dst, &g->ioff, &g->inbr);  /* in-neighbours */
        return g;
    }
    /* adjacency lists: both directions, then sort and drop repeats and loops */
    int64_t *deg = calloc(nv + 1, sizeof *deg);
    for (int64_t e = 0; e < ne; e++)
        if (src[e] != dst[e]) { deg[src[e]]++; deg[dst[e]]++; }
    int64_t *start = malloc((nv + 1) * sizeof *start);
    start[0] = 0;
    for (int64_t v = 0; v < nv; v++) start[v + 1] = start[v] + deg[v];
    int32_t *tmp = malloc((start[nv] > 0 ? start[nv] : 1) * sizeof *tmp);
    int64_t *fill = calloc(nv + 1, sizeof *fill);
    for (int64_t e = 0; e < ne; e++) {
        if (src[e] == dst[e]) continue;
        tmp[start[src[e]] + fill[src[e]]++] = dst[e];
        tmp[start[dst[e]] + fill[dst[e]]++] = src[e];
    }
    g->off = malloc((nv + 1) * sizeof *g->off);
    g->nbr = malloc((start[nv] > 0 ? start[nv] : 1) * sizeof *g->nbr);
    int64_t k = 0;
    for (int64_t v = 0; v < nv; v++) {
        g->off[v] = k;
        int32_t *row = tmp + start[v];
        qsort(row, (size_t)deg[v], sizeof *row, cmp_i32);
        for (int64_t i = 0; i < deg[v]; i++)
            if (i == 0 || row[i] != row[i - 1]) g->nbr[k++] = row[i];
    }
    g->off[nv] = k;
    free(deg); free(start); free(tmp); free(fill);
    return g;
}

void *or_graph_new(int64_t nv, const int32_t *labels, int64_t ne, const int32_t *src,
                   const int32_t *dst, uint64_t seed)
{
    return or_graph_new2(nv, labels, ne, src, dst, seed, 0);
}

/* Root-order variant of R4: id_order = 1 visits roots by vertex id, 0 by (H(seed, v), v). */
void or_graph_set_root_order(void *gp, int id_order)
{
    ((or_graph *)gp)->id_order = id_order ? 1 : 0;
}

void or_graph_free(void *gp)
{
    or_graph *g = gp;
    if (!g) return;
    free(g->rank_of); free(g->lab); free(g->off); free(g->nbr); free(g->ioff); free(g->inbr); free(g);
}

int64_t or_graph_arcs(void *gp) { return ((or_graph *)gp)->off[((or_graph *)gp)->nv]; }
int32_t or_graph_rank(void *gp, int32_t label)
{
    or_graph *g = gp;
    return (label < 0 || label >= g->nl) ? -1 : g->rank_of[label];
}

/* an edge u - v (undirected) or an arc u -> v (directed) */
static int adjacent(const or_graph *g, int32_t u, int32_t v)
{
    int64_t lo = g->off[u], hi = g->off[u + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (g->nbr[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < g->off[u + 1] && g->nbr[lo] == v;
}

/* ------------------------------------------------------------------ patterns, R2 canonical form
 * A small pattern: n <= 8 vertices, labels lab[n], adjacency matrix adj[n][n]: symmetric for an
 * undirected pattern, adj[i][j] = arc i -> j for a directed one.                               */
typedef struct {
    int n;
    int directed;
    int32_t lab[OR_MAXN];
    uint8_t adj[OR_MAXN][OR_MAXN];
} or_pat;

/* i and j joined by an edge or an arc either way */
static int linked(const or_pat *p, int i, int j) { return p->adj[i][j] || p->adj[j][i]; }

/* code of the pattern read in the vertex order perm[0..n-1] (position p holds vertex perm[p]).
 * Undirected: for j = 1..n-1, i = 0..j-1 the bit "i not adjacent to j".  Directed (R2 for
 * directed patterns): for each such pair two bits, "no arc i -> j" then "no arc j -> i".       */
typedef struct {
    int n;
    int32_t lab[OR_MAXN];
    uint64_t bits;       /* first code bit is the most significant one */
} or_code;

static or_code code_of(const or_pat *p, const int *perm)
{
    or_code c;
    memset(&c, 0, sizeof c);
    c.n = p->n;
    for (int i = 0; i < p->n; i++) c.lab[i] = p->lab[perm[i]];
    uint64_t bits = 0;
    for (int j = 1; j < p->n; j++)
        for (int i = 0; i < j; i++) {
            bits = (bits << 1) | (p->adj[perm[i]][perm[j]] ? 0u : 1u);
            if (p->directed) bits = (bits << 1) | (p->adj[perm[j]][perm[i]] ? 0u : 1u);
        }
    c.bits = bits;
    return c;
}

static int code_cmp(const or_code *a, const or_code *b)
{
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = 0; i < a->n; i++)
        if (a->lab[i] != b->lab[i]) return a->lab[i] < b->lab[i] ? -1 : 1;
    if (a->bits != b->bits) return a->bits < b->bits ? -1 : 1;
    return 0;
}

/* brute force: every one of the n! orders */
static void canon_rec(const or_pat *p, int *perm, int pos, int used, or_code *best, int *best_perm,
                      int *have)
{
    if (pos == p->n) {
        or_code c = code_of(p, perm);
        if (!*have || code_cmp(&c, best) < 0) {
            *best = c;
            memcpy(best_perm, perm, sizeof(int) * p->n);
            *have = 1;
        }
        return;
    }
    for (int v = 0; v < p->n; v++) {
        if (used & (1 << v)) continue;
        perm[pos] = v;
        canon_rec(p, perm, pos + 1, used | (1 << v), best, best_perm, have);
    }
}

/* canonical pattern: position p of the result is vertex perm[p] of the input */
static or_pat canonical(const or_pat *p, int *perm_out)
{
    int perm[OR_MAXN], best_perm[OR_MAXN], have = 0;
    or_code best;
    memset(&best, 0, sizeof best);
    canon_rec(p, perm, 0, 0, &best, best_perm, &have);
    or_pat q;
    memset(&q, 0, sizeof q);
    q.n = p->n;
    q.directed = p->directed;
    for (int i = 0; i < p->n; i++) {
        q.lab[i] = p->lab[best_perm[i]];
        for (int j = 0; j < p->n; j++) q.adj[i][j] = p->adj[best_perm[i]][best_perm[j]];
    }
    if (perm_out) memcpy(perm_out, best_perm, sizeof(int) * p->n);
    return q;
}

static int pat_connected(const or_pat *p)
{
    int seen = 1, grew = 1;
    while (grew) {
        grew = 0;
        for (int u = 0; u < p->n; u++)
            if (seen & (1 << u))
                for (int v = 0; v < p->n; v++)
                    if (linked(p, u, v) && !(seen & (1 << v))) { seen |= 1 << v; grew = 1; }
    }
    return seen == (1 << p->n) - 1;
}

static int pat_edges(const or_pat *p)
{
    int m = 0;
    for (int i = 0; i < p->n; i++)
        for (int j = i + 1; j < p->n; j++) m += p->adj[i][j];
    return m;
}

/* build from (labels, edge list); a directed pattern takes each edge (a, b) as the arc a -> b.
 * Returns -1 on a bad edge. */
static int pat_from_dir(or_pat *p, int n, const int32_t *labels, int m, const int32_t *edges, int directed)
{
    if (n < 1 || n > OR_MAXN) return -1;
    memset(p, 0, sizeof *p);
    p->n = n;
    p->directed = directed ? 1 : 0;
    for (int i = 0; i < n; i++) p->lab[i] = labels[i];
    for (int e = 0; e < m; e++) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) return -1;
        p->adj[a][b] = 1;
        if (!directed) p->adj[b][a] = 1;
    }
    return 0;
}

static int pat_from(or_pat *p, int n, const int32_t *labels, int m, const int32_t *edges)
{
    return pat_from_dir(p, n, labels, m, edges, 0);
}

/* exported: canonical code of a pattern whose labels are used as given.
 * out_labels[n], out_bits, out_perm[n] (position -> input vertex).                              */
int or_canonical(int n, const int32_t *labels, int m, const int32_t *edges, int32_t *out_labels,
                 uint32_t *out_bits, int32_t *out_perm)
{
    or_pat p;
    if (pat_from(&p, n, labels, m, edges)) return -1;
    int perm[OR_MAXN];
    or_pat q = canonical(&p, perm);
    int id[OR_MAXN];
    for (int i = 0; i < n; i++) id[i] = i;
    or_code c = code_of(&q, id);
    for (int i = 0; i < n; i++) { out_labels[i] = c.lab[i]; if (out_perm) out_perm[i] = perm[i]; }
    *out_bits = (uint32_t)c.bits;
    return 0;
}

/* R3 matching order starting at canonical position `first` */
static void matching_order(const or_pat *q, int first, int *pi)
{
    int visited = 1 << first;
    pi[0] = first;
    for (int k = 1; k < q->n; k++) {
        int pick = -1;
        for (int v = 0; v < q->n && pick < 0; v++) {
            if (visited & (1 << v)) continue;
            for (int u = 0; u < q->n; u++)
                if ((visited & (1 << u)) && linked(q, u, v)) { pick = v; break; }
        }
        pi[k] = pick;           /* q is connected, so pick >= 0 */
        visited |= 1 << pick;
    }
}

/* ------------------------------------------------------------------ maps, Sec. 2.1.4 / 2.4
 * A map e sends canonical pattern vertex i to data vertex e[i]: injective, label preserving,
 * and every pattern edge lands on a data edge (non-induced).                                   */
typedef struct {
    int32_t v[OR_MAXN];
} or_map;

typedef struct {
    or_map *a;
    int64_t len, cap;
} map_list;

static void ml_push(map_list *l, const int32_t *v, int n)
{
    if (l->len == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 64;
        l->a = realloc(l->a, (size_t)l->cap * sizeof *l->a);
    }
    memset(&l->a[l->len], 0, sizeof(or_map));
    memcpy(l->a[l->len].v, v, sizeof(int32_t) * n);
    l->len++;
}

static int is_map(const or_graph *g, const or_pat *q, const int32_t *e)
{
    for (int i = 0; i < q->n; i++) {
        if (g->lab[e[i]] != q->lab[i]) return 0;
        for (int j = 0; j < i; j++) {
            if (e[i] == e[j]) return 0;
            if (q->adj[i][j] && !adjacent(g, e[i], e[j])) return 0;
            if (q->adj[j][i] && !adjacent(g, e[j], e[i])) return 0;
        }
    }
    return 1;
}

/* tier 0: every tuple of V^n, in order */
static void maps_brute(const or_graph *g, const or_pat *q, map_list *out)
{
    int32_t e[OR_MAXN] = {0};
    int n = q->n;
    for (;;) {
        if (is_map(g, q, e)) ml_push(out, e, n);
        int k = n - 1;
        while (k >= 0 && ++e[k] == g->nv) { e[k] = 0; k--; }
        if (k < 0) break;
    }
}

/* sort key R4 */
static const int *g_pi;
static uint64_t g_seed;
static int g_id_order;
static int g_n;

static uint64_t root_key(int32_t r) { return g_id_order ? 0 : or_hash(g_seed, r); }

static int cmp_map_key(const void *pa, const void *pb)
{
    const or_map *a = pa, *b = pb;
    int32_t ra = a->v[g_pi[0]], rb = b->v[g_pi[0]];
    uint64_t ha = root_key(ra), hb = root_key(rb);
    if (ha != hb) return ha < hb ? -1 : 1;
    if (ra != rb) return ra < rb ? -1 : 1;
    for (int k = 1; k < g_n; k++) {
        int32_t x = a->v[g_pi[k]], y = b->v[g_pi[k]];
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ tier 1: backtracking
 * Depth-first over the matching order; candidates for level k are the neighbours (ascending
 * id) of the data vertex at the first earlier level adjacent to pi_k.  `used` (nullable) marks
 * vertices that may not appear.  Returns 1 at the first complete map when stop_first, else
 * collects all maps into `out`.                                                                 */
typedef struct {
    const or_graph *g;
    const or_pat *q;
    const int *pi;
    const uint8_t *used;
    int stop_first;
    map_list *out;
    int64_t count;
    int64_t count_cap;
    int64_t *nodes;      /* nullable: candidates tried, shared by every search of one call */
    int64_t budget;      /* > 0: give up once *nodes passes it (the call is then skipped) */
    int *aborted;
    int32_t e[OR_MAXN];
} bt_state;

static int bt_level(bt_state *s, int k)
{
    const or_graph *g = s->g;
    const or_pat *q = s->q;
    int n = q->n;
    if (k == n) {
        s->count++;
        if (s->out) ml_push(s->out, s->e, n);
        return s->stop_first || (s->count_cap > 0 && s->count >= s->count_cap);
    }
    int vk = s->pi[k];
    int anchor = -1;
    for (int j = 0; j < k && anchor < 0; j++)
        if (linked(q, s->pi[j], vk)) anchor = s->pi[j];
    int32_t a = s->e[anchor];
    /* candidates: out-neighbours of the anchor's image for an arc anchor -> vk (all neighbours
     * when undirected), else its in-neighbours */
    const int64_t *off = g->off;
    const int32_t *nbr = g->nbr;
    if (g->directed && !q->adj[anchor][vk]) { off = g->ioff; nbr = g->inbr; }
    for (int64_t t = off[a]; t < off[a + 1]; t++) {
        int32_t c = nbr[t];
        if (s->nodes && ++*s->nodes > s->budget) { *s->aborted = 1; return 1; }
        if (g->lab[c] != q->lab[vk]) continue;
        if (s->used && s->used[c]) continue;
        int ok = 1;
        for (int j = 0; j < k && ok; j++) {
            int vj = s->pi[j];
            if (s->e[vj] == c) ok = 0;
            else if (q->adj[vj][vk] && !adjacent(g, s->e[vj], c)) ok = 0;
            else if (q->adj[vk][vj] && !adjacent(g, c, s->e[vj])) ok = 0;
        }
        if (!ok) continue;
        s->e[vk] = c;
        if (bt_level(s, k + 1)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ support evaluation
 * out[0..7]: tau, mis, mni, n_maps (tier 0 only, else -1), frequent, n, cap, status.
 * mode 0 = FULL (exact counts), 1 = EARLY (counts capped at c = max(tau, 1)), 2 = EARLY without
 * the MNI count (mni = -1: the metric step of Sec. 3.2.2 computes the mIS only).
 * tier 0 = brute force over V^n with an explicit sorted map list; tier 1 = backtracking.
 * sel_out (nullable, capacity sel_cap maps of 8 ids) receives the selected maps, as
 * canonical-vertex-indexed tuples; *n_sel their number.
 * budget > 0 (tier 1): give up after that many candidate vertices tried over all searches of the
 * call and return -3 (the pattern is skipped, nothing is reported).                             */
int or_support_budget(void *gp, int n, const int32_t *labels, int m, const int32_t *edges, int64_t sigma,
                      int64_t lam_num, int64_t lam_den, int mode, int tier, int64_t *out,
                      int32_t *sel_out, int64_t sel_cap, int64_t *n_sel, int64_t budget)
{
    const or_graph *g = gp;
    int64_t nodes = 0;
    int aborted = 0;
    const int want_mni = mode != 2;
    if (mode == 2) mode = 1;
    memset(out, 0, 8 * sizeof *out);
    if (n_sel) *n_sel = 0;
    if (n < 2 || n > OR_MAXN || sigma < 1 || lam_den <= 0 || lam_num < 0 || lam_num > lam_den)
        return -1;
    or_pat p;
    if (pat_from_dir(&p, n, labels, m, edges, g->directed)) return -1;
    for (int i = 0; i < n; i++) if (labels[i] < 0) return -1;
    if (!pat_connected(&p)) return -1;
    int64_t tau = or_tau(sigma, lam_num, lam_den, n);
    int64_t cap = tau > 1 ? tau : 1;
    out[0] = tau;
    out[5] = n;
    out[6] = mode == 1 ? cap : -1;
    out[3] = tier == 0 ? 0 : -1;
    /* a label with no data vertex: no map at all */
    for (int i = 0; i < n; i++) {
        int32_t r = (labels[i] < g->nl) ? g->rank_of[labels[i]] : -1;
        if (r < 0) return 0;
        p.lab[i] = r;
    }
    or_pat q = canonical(&p, NULL);
    int pi[OR_MAXN];
    matching_order(&q, 0, pi);

    int64_t mis = 0, mni = 0;
    uint8_t *used = calloc(g->nv > 0 ? g->nv : 1, 1);
    if (tier == 0) {
        map_list M = {0};
        maps_brute(g, &q, &M);
        out[3] = M.len;
        g_pi = pi; g_seed = g->seed; g_id_order = g->id_order; g_n = n;
        qsort(M.a, (size_t)M.len, sizeof *M.a, cmp_map_key);
        /* sequential greedy over the ordered list: keep a map iff none of its vertices is used */
        for (int64_t t = 0; t < M.len; t++) {
            int free_ = 1;
            for (int i = 0; i < n; i++) if (used[M.a[t].v[i]]) free_ = 0;
            if (!free_) continue;
            for (int i = 0; i < n; i++) used[M.a[t].v[i]] = 1;
            if (sel_out && mis < sel_cap) memcpy(sel_out + 8 * mis, M.a[t].v, 8 * sizeof(int32_t));
            mis++;
        }
        /* MNI, Sec. 2.4.4: min over pattern vertices of the number of distinct images */
        uint8_t *seen = calloc(g->nv > 0 ? g->nv : 1, 1);
        mni = -1;
        for (int u = 0; u < n; u++) {
            memset(seen, 0, (size_t)g->nv);
            int64_t f = 0;
            for (int64_t t = 0; t < M.len; t++)
                if (!seen[M.a[t].v[u]]) { seen[M.a[t].v[u]] = 1; f++; }
            if (mni < 0 || f < mni) mni = f;
        }
        free(seen);
        free(M.a);
        if (mode == 1) { if (mis > cap) mis = cap; if (mni > cap) mni = cap; }
        if (!want_mni) mni = -1;
    } else {
        /* roots = vertices carrying the label of pi_0, in (H, id) order */
        int64_t nr = 0;
        for (int64_t v = 0; v < g->nv; v++) if (g->lab[v] == q.lab[pi[0]]) nr++;
        int32_t *roots = malloc((nr > 0 ? nr : 1) * sizeof *roots);
        nr = 0;
        for (int64_t v = 0; v < g->nv; v++) if (g->lab[v] == q.lab[pi[0]]) roots[nr++] = (int32_t)v;
        /* insertion into (hash, id) order by a plain sort */
        or_map *tmp = malloc((nr > 0 ? nr : 1) * sizeof *tmp);
        for (int64_t i = 0; i < nr; i++) { memset(&tmp[i], 0, sizeof tmp[i]); tmp[i].v[pi[0]] = roots[i]; }
        g_pi = pi; g_seed = g->seed; g_id_order = g->id_order; g_n = 1; /* compare by root only */
        qsort(tmp, (size_t)nr, sizeof *tmp, cmp_map_key);
        for (int64_t i = 0; i < nr; i++) roots[i] = tmp[i].v[pi[0]];
        free(tmp);
        /* Sec. 3.2.2: for each root in order, the first map (lexicographic in matching order)
         * avoiding used vertices is selected; the search of that root then stops.            */
        for (int64_t i = 0; i < nr; i++) {
            if (mode == 1 && mis >= cap) break;
            int32_t r = roots[i];
            if (used[r]) continue;
            bt_state s;
            memset(&s, 0, sizeof s);
            s.g = g; s.q = &q; s.pi = pi; s.used = used; s.stop_first = 1;
            if (budget > 0) { s.nodes = &nodes; s.budget = budget; s.aborted = &aborted; }
            s.e[pi[0]] = r;
            const int hit = bt_level(&s, 1);
            if (aborted) break;
            if (hit) {
                for (int k = 0; k < n; k++) used[s.e[k]] = 1;
                if (sel_out && mis < sel_cap) memcpy(sel_out + 8 * mis, s.e, 8 * sizeof(int32_t));
                mis++;
            }
        }
        free(roots);
        /* MNI: for every pattern vertex u and every data vertex d with u's label, is there a map
         * with u -> d?  (matching order rooted at u; stop at the first hit)                   */
        mni = -1;
        for (int u = 0; u < n && want_mni && !aborted; u++) {
            int piu[OR_MAXN];
            matching_order(&q, u, piu);
            int64_t f = 0;
            for (int64_t d = 0; d < g->nv; d++) {
                if (g->lab[d] != q.lab[u]) continue;
                if (mode == 1 && f >= cap) break;
                bt_state s;
                memset(&s, 0, sizeof s);
                s.g = g; s.q = &q; s.pi = piu; s.used = NULL; s.stop_first = 1;
                if (budget > 0) { s.nodes = &nodes; s.budget = budget; s.aborted = &aborted; }
                s.e[u] = (int32_t)d;
                const int hit = bt_level(&s, 1);
                if (aborted) break;
                if (hit) f++;
            }
            if (mni < 0 || f < mni) mni = f;
        }
        if (!want_mni) mni = -1;
    }
    free(used);
    if (aborted) return -3;
    out[1] = mis;
    out[2] = mni;
    out[4] = mis >= cap ? 1 : 0;
    if (n_sel) *n_sel = mis < sel_cap ? mis : sel_cap;
    return 0;
}

int or_support(void *gp, int n, const int32_t *labels, int m, const int32_t *edges, int64_t sigma,
               int64_t lam_num, int64_t lam_den, int mode, int tier, int64_t *out,
               int32_t *sel_out, int64_t sel_cap, int64_t *n_sel)
{
    return or_support_budget(gp, n, labels, m, edges, sigma, lam_num, lam_den, mode, tier, out, sel_out,
                             sel_cap, n_sel, 0);
}

/* count of all maps by backtracking (tier 1), stopping at count_cap if > 0 */
int64_t or_count_maps(void *gp, int n, const int32_t *labels, int m, const int32_t *edges,
                      int64_t count_cap)
{
    const or_graph *g = gp;
    or_pat p;
    if (pat_from_dir(&p, n, labels, m, edges, g->directed) || !pat_connected(&p)) return -1;
    for (int i = 0; i < n; i++) {
        int32_t r = (labels[i] >= 0 && labels[i] < g->nl) ? g->rank_of[labels[i]] : -1;
        if (r < 0) return 0;
        p.lab[i] = r;
    }
    or_pat q = canonical(&p, NULL);
    int pi[OR_MAXN];
    matching_order(&q, 0, pi);
    int64_t total = 0;
    for (int64_t r = 0; r < g->nv; r++) {
        if (g->lab[r] != q.lab[pi[0]]) continue;
        bt_state s;
        memset(&s, 0, sizeof s);
        s.g = g; s.q = &q; s.pi = pi; s.count_cap = count_cap > 0 ? count_cap - total : 0;
        s.e[pi[0]] = (int32_t)r;
        bt_level(&s, 1);
        total += s.count;
        if (count_cap > 0 && total >= count_cap) break;
    }
    return total;
}

/* ------------------------------------------------------------------ overlap graph and MIS
 * Sec. 2.4.1: two maps overlap when they share a data vertex.  Maps with the same image vertex
 * set (an "instance") overlap each other and every other map the same way, so a maximum
 * independent set of maps (Sec. 2.4.2) has the size of a maximum independent set of distinct
 * instances.  The oracle lists every map (tier-1 backtracking, no used set), sorts each map's
 * image ascending, sorts and deduplicates the instances, and joins two instances by a conflict
 * edge when their vertex sets intersect (plain pairwise test).                                 */
static int cmp_inst(const void *a, const void *b)
{
    const int32_t *x = a, *y = b;
    for (int i = 0; i < OR_MAXN; i++)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

/* instances (sorted rows of 8 ids, -1 padded) of a pattern; returns their number, -1 on a bad
 * pattern, or -2 if the pattern has more than max_maps maps.  *out is malloc'ed.               */
static int64_t instances_of(const or_graph *g, int n, const int32_t *labels, int m, const int32_t *edges,
                            int64_t max_maps, int32_t **out)
{
    *out = NULL;
    or_pat p;
    if (n < 2 || pat_from_dir(&p, n, labels, m, edges, g->directed) || !pat_connected(&p)) return -1;
    for (int i = 0; i < n; i++) {
        int32_t r = (labels[i] >= 0 && labels[i] < g->nl) ? g->rank_of[labels[i]] : -1;
        if (r < 0) return 0;
        p.lab[i] = r;
    }
    or_pat q = canonical(&p, NULL);
    int pi[OR_MAXN];
    matching_order(&q, 0, pi);
    map_list M = {0};
    for (int64_t r = 0; r < g->nv; r++) {
        if (g->lab[r] != q.lab[pi[0]]) continue;
        bt_state s;
        memset(&s, 0, sizeof s);
        s.g = g; s.q = &q; s.pi = pi; s.out = &M;
        s.e[pi[0]] = (int32_t)r;
        bt_level(&s, 1);
        if (M.len > max_maps) { free(M.a); return -2; }
    }
    int32_t *rows = malloc((M.len > 0 ? M.len : 1) * OR_MAXN * sizeof *rows);
    for (int64_t t = 0; t < M.len; t++) {
        int32_t *row = rows + OR_MAXN * t;
        for (int i = 0; i < OR_MAXN; i++) row[i] = i < n ? M.a[t].v[i] : -1;
        /* insertion sort of the n image vertices */
        for (int i = 1; i < n; i++)
            for (int k = i; k > 0 && row[k - 1] > row[k]; k--) { int32_t x = row[k]; row[k] = row[k - 1]; row[k - 1] = x; }
    }
    free(M.a);
    qsort(rows, (size_t)M.len, OR_MAXN * sizeof *rows, cmp_inst);
    int64_t k = 0;
    for (int64_t t = 0; t < M.len; t++)
        if (k == 0 || cmp_inst(rows + OR_MAXN * t, rows + OR_MAXN * (k - 1)) != 0) {
            if (k != t) memcpy(rows + OR_MAXN * k, rows + OR_MAXN * t, OR_MAXN * sizeof *rows);
            k++;
        }
    *out = rows;
    return k;
}

static int inst_meet(const int32_t *a, const int32_t *b, int n)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) if (a[i] == b[j]) return 1;
    return 0;
}

/* exported: the overlap graph of a pattern's instances.  inst_out[cap_inst * 8] (sorted,
 * -1 padded rows, in ascending order), *n_inst; edges_out[2 * cap_edges] pairs a < b in
 * lexicographic order, *n_edges.  Returns 0, -1 on a bad pattern, -2 if the maps exceed
 * max_maps or the instances / edges exceed their capacities.                                  */
int or_overlap_graph(void *gp, int n, const int32_t *labels, int m, const int32_t *edges, int64_t max_maps,
                     int32_t *inst_out, int64_t cap_inst, int64_t *n_inst, int32_t *edges_out,
                     int64_t cap_edges, int64_t *n_edges)
{
    int32_t *rows;
    int64_t k = instances_of(gp, n, labels, m, edges, max_maps, &rows);
    *n_inst = k > 0 ? k : 0;
    *n_edges = 0;
    if (k < 0) { free(rows); return (int)k; }
    if (k > cap_inst) { free(rows); return -2; }
    if (k > 0) memcpy(inst_out, rows, (size_t)k * OR_MAXN * sizeof *rows);
    int64_t e = 0;
    for (int64_t a = 0; a < k; a++)
        for (int64_t b = a + 1; b < k; b++)
            if (inst_meet(rows + OR_MAXN * a, rows + OR_MAXN * b, n)) {
                if (e >= cap_edges) { free(rows); return -2; }
                edges_out[2 * e] = (int32_t)a;
                edges_out[2 * e + 1] = (int32_t)b;
                e++;
            }
    *n_edges = e;
    free(rows);
    return 0;
}

/* maximum independent set of the instances (Sec. 2.4.2) by exhaustive search: each instance is
 * either taken (if it meets no taken one) or left out; a branch stops when even taking every
 * remaining instance could not beat the best set found.                                        */
typedef struct {
    const int32_t *rows;
    int n;
    int64_t k;
    uint8_t *conf;   /* k x k conflict matrix */
    int64_t best;
} mis_state;

static void mis_rec(mis_state *s, int64_t i, int64_t size, uint8_t *taken)
{
    if (size + (s->k - i) <= s->best) return;
    if (i == s->k) { s->best = size; return; }
    int ok = 1;
    for (int64_t j = 0; j < i && ok; j++)
        if (taken[j] && s->conf[i * s->k + j]) ok = 0;
    if (ok) {
        taken[i] = 1;
        mis_rec(s, i + 1, size + 1, taken);
        taken[i] = 0;
    }
    mis_rec(s, i + 1, size, taken);
}

/* exported: size of a maximum independent set of the pattern's maps; -1 on a bad pattern, -2 if
 * the maps exceed max_maps or the instances exceed max_inst.                                   */
int64_t or_max_independent_set(void *gp, int n, const int32_t *labels, int m, const int32_t *edges,
                               int64_t max_maps, int64_t max_inst)
{
    int32_t *rows;
    int64_t k = instances_of(gp, n, labels, m, edges, max_maps, &rows);
    if (k < 0) { free(rows); return k; }
    if (k > max_inst) { free(rows); return -2; }
    mis_state s;
    s.rows = rows; s.n = n; s.k = k; s.best = 0;
    s.conf = calloc((size_t)(k > 0 ? k * k : 1), 1);
    for (int64_t a = 0; a < k; a++)
        for (int64_t b = 0; b < k; b++)
            s.conf[a * k + b] = (uint8_t)(a != b && inst_meet(rows + OR_MAXN * a, rows + OR_MAXN * b, n));
    uint8_t *taken = calloc((size_t)(k > 0 ? k : 1), 1);
    mis_rec(&s, 0, 0, taken);
    free(taken); free(s.conf); free(rows);
    return s.best;
}

/* ------------------------------------------------------------------ candidate generation
 * Predicate form of Algorithms 2-4 (Sec. 3.2.1).  With F = the frequent (k-1)-vertex patterns,
 * a connected k-vertex pattern P is a candidate iff
 *   (i)  P is not a clique and there are two NON-adjacent vertices u != v with P-u and P-v both
 *        isomorphic to members of F  (what merging two core graphs on a common core yields,
 *        Lemma 3: the two marked vertices stay non-adjacent), or
 *   (ii) P is a clique and every P-u is in F  (three-clique merge plus the post-check that all
 *        (k-1)-sub-cliques are frequent, Lemma 4).
 * The oracle enumerates every one-vertex extension of every member of F (each label seen in F,
 * each non-empty set of attachment vertices), keeps those satisfying the predicate and removes
 * duplicates by canonical code.  Labels are used as given (no ranking).                         */
typedef struct {
    or_code *a;
    int64_t len, cap;
} code_set;

static int64_t cs_find(const code_set *s, const or_code *c)
{
    for (int64_t i = 0; i < s->len; i++) if (code_cmp(&s->a[i], c) == 0) return i;
    return -1;
}

static void cs_add(code_set *s, const or_code *c)
{
    if (cs_find(s, c) >= 0) return;
    if (s->len == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 64;
        s->a = realloc(s->a, (size_t)s->cap * sizeof *s->a);
    }
    s->a[s->len++] = *c;
}

static or_code canon_code(const or_pat *p)
{
    or_pat q = canonical(p, NULL);
    int id[OR_MAXN];
    for (int i = 0; i < q.n; i++) id[i] = i;
    return code_of(&q, id);
}

static or_pat pat_of_code(const or_code *c)
{
    or_pat p;
    memset(&p, 0, sizeof p);
    p.n = c->n;
    for (int i = 0; i < c->n; i++) p.lab[i] = c->lab[i];
    int t = c->n * (c->n - 1) / 2 - 1;
    for (int j = 1; j < c->n; j++)
        for (int i = 0; i < j; i++, t--) {
            int nonadj = (c->bits >> t) & 1;
            p.adj[i][j] = p.adj[j][i] = nonadj ? 0 : 1;
        }
    return p;
}

static or_pat pat_minus(const or_pat *p, int u)
{
    or_pat r;
    memset(&r, 0, sizeof r);
    r.n = p->n - 1;
    int map[OR_MAXN], k = 0;
    for (int i = 0; i < p->n; i++) if (i != u) map[k++] = i;
    for (int i = 0; i < r.n; i++) {
        r.lab[i] = p->lab[map[i]];
        for (int j = 0; j < r.n; j++) r.adj[i][j] = p->adj[map[i]][map[j]];
    }
    return r;
}

/* sub-pattern P-u is "in F": connected and its canonical code is a member */
static int minus_in(const or_pat *p, int u, const code_set *F)
{
    or_pat r = pat_minus(p, u);
    if (!pat_connected(&r)) return 0;
    or_code c = canon_code(&r);
    return cs_find(F, &c) >= 0;
}

static int is_candidate(const or_pat *p, const code_set *F)
{
    int n = p->n, clique = 1;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) if (!p->adj[i][j]) clique = 0;
    if (clique) {
        for (int u = 0; u < n; u++) if (!minus_in(p, u, F)) return 0;
        return 1;
    }
    int in[OR_MAXN];
    for (int u = 0; u < n; u++) in[u] = minus_in(p, u, F);
    for (int u = 0; u < n; u++)
        for (int v = u + 1; v < n; v++)
            if (!p->adj[u][v] && in[u] && in[v]) return 1;
    return 0;
}

static void gen_candidates(const code_set *F, int max_edges, code_set *out)
{
    int32_t labs[256];
    int nlabs = 0;
    for (int64_t f = 0; f < F->len; f++)
        for (int i = 0; i < F->a[f].n; i++) {
            int seen = 0;
            for (int t = 0; t < nlabs; t++) if (labs[t] == F->a[f].lab[i]) seen = 1;
            if (!seen && nlabs < 256) labs[nlabs++] = F->a[f].lab[i];
        }
    for (int64_t f = 0; f < F->len; f++) {
        or_pat base = pat_of_code(&F->a[f]);
        int k = base.n;
        if (k + 1 > OR_MAXN) continue;
        for (int li = 0; li < nlabs; li++)
            for (int S = 1; S < (1 << k); S++) {
                or_pat p = base;
                p.n = k + 1;
                p.lab[k] = labs[li];
                for (int i = 0; i < k; i++) {
                    int a = (S >> i) & 1;
                    p.adj[i][k] = p.adj[k][i] = (uint8_t)a;
                }
                p.adj[k][k] = 0;
                if (max_edges > 0 && pat_edges(&p) > max_edges) continue;
                if (!is_candidate(&p, F)) continue;
                or_code c = canon_code(&p);
                cs_add(out, &c);
            }
    }
}

static int cmp_code_q(const void *a, const void *b) { return code_cmp(a, b); }

/* exported: candidates from a list of frequent (k-1)-vertex patterns (given as label/edge
 * lists).  Writes canonical codes (n, labels[8], bits) of the candidates, sorted, into
 * out_n[cap], out_lab[cap*8], out_bits[cap]; returns their number (or -needed if > cap).       */
int64_t or_candidates(int count, const int32_t *ns, const int32_t *labels /* count*8 */,
                      const int32_t *ms, const int32_t *edges /* count*2*28 */, int max_edges,
                      int32_t *out_n, int32_t *out_lab, uint32_t *out_bits, int64_t cap)
{
    code_set F = {0}, C = {0};
    for (int i = 0; i < count; i++) {
        or_pat p;
        if (pat_from(&p, ns[i], labels + 8 * i, ms[i], edges + 56 * i)) { free(F.a); return -1; }
        or_code c = canon_code(&p);
        cs_add(&F, &c);
    }
    gen_candidates(&F, max_edges, &C);
    qsort(C.a, (size_t)C.len, sizeof *C.a, cmp_code_q);
    int64_t n = C.len;
    if (n <= cap)
        for (int64_t i = 0; i < n; i++) {
            out_n[i] = C.a[i].n;
            for (int j = 0; j < 8; j++) out_lab[8 * i + j] = j < C.a[i].n ? C.a[i].lab[j] : 0;
            out_bits[i] = (uint32_t)C.a[i].bits;
        }
    free(F.a); free(C.a);
    return n <= cap ? n : -n;
}

/* ------------------------------------------------------------------ mining, Algorithm 1
 * Level 2 candidates are the label pairs found on data edges (edges(G)); then level by level:
 * evaluate every candidate (tier 1, EARLY mode), keep the frequent ones, generate the next
 * candidates from them.  Levels are counted in vertices; only candidates with at most
 * max_edges edges are kept, so levels run k = 2 .. max_edges + 1.                              */
typedef struct {
    int64_t len, cap;
    or_code *code;       /* rank-space canonical codes */
    int64_t *res;        /* [len][4]: tau, mis, mni, frequent */
    int64_t lvl_cand[OR_MAXN + 1], lvl_freq[OR_MAXN + 1];
} or_mined;

static void mined_push(or_mined *r, const or_code *c, const int64_t *o)
{
    if (r->len == r->cap) {
        r->cap = r->cap ? 2 * r->cap : 64;
        r->code = realloc(r->code, (size_t)r->cap * sizeof *r->code);
        r->res = realloc(r->res, (size_t)r->cap * 4 * sizeof *r->res);
    }
    r->code[r->len] = *c;
    r->res[4 * r->len + 0] = o[0];
    r->res[4 * r->len + 1] = o[1];
    r->res[4 * r->len + 2] = o[2];
    r->res[4 * r->len + 3] = o[4];
    r->len++;
}

/* evaluate a rank-space canonical pattern (labels are ranks, so translate back to ids) */
static void eval_code(const or_graph *g, const or_code *c, int64_t sigma, int64_t ln, int64_t ld,
                      int64_t *o)
{
    or_pat p = pat_of_code(c);
    int32_t labels[OR_MAXN], edges[2 * 28];
    int m = 0;
    for (int i = 0; i < p.n; i++) {
        for (int32_t a = 0; a < g->nl; a++) if (g->rank_of[a] == p.lab[i]) labels[i] = a;
        for (int j = i + 1; j < p.n; j++)
            if (p.adj[i][j]) { edges[2 * m] = i; edges[2 * m + 1] = j; m++; }
    }
    /* the metric step computes the mIS decision (Sec. 3.2.2); for a frequent pattern the MNI,
     * capped at c, is c (mIS <= MNI), which is what is recorded */
    or_support((void *)g, p.n, labels, m, edges, sigma, ln, ld, 2, 1, o, NULL, 0, NULL);
    if (o[4]) o[2] = o[6];
}

void *or_mine(void *gp, int64_t sigma, int64_t lam_num, int64_t lam_den, int max_edges)
{
    const or_graph *g = gp;
    or_mined *r = calloc(1, sizeof *r);
    code_set C = {0}, F = {0};
    /* edges(G): one candidate per label pair present on a data edge */
    for (int64_t u = 0; u < g->nv; u++)
        for (int64_t t = g->off[u]; t < g->off[u + 1]; t++) {
            or_pat p;
            memset(&p, 0, sizeof p);
            p.n = 2;
            p.lab[0] = g->lab[u];
            p.lab[1] = g->lab[g->nbr[t]];
            p.adj[0][1] = p.adj[1][0] = 1;
            or_code c = canon_code(&p);
            cs_add(&C, &c);
        }
    for (int k = 2; k <= max_edges + 1 && k <= OR_MAXN && C.len > 0; k++) {
        qsort(C.a, (size_t)C.len, sizeof *C.a, cmp_code_q);
        F.len = 0;
        r->lvl_cand[k] = C.len;
        for (int64_t i = 0; i < C.len; i++) {
            int64_t o[8];
            eval_code(g, &C.a[i], sigma, lam_num, lam_den, o);
            if (o[4]) { cs_add(&F, &C.a[i]); mined_push(r, &C.a[i], o); }
        }
        r->lvl_freq[k] = F.len;
        C.len = 0;
        if (k + 1 <= max_edges + 1) gen_candidates(&F, max_edges, &C);
    }
    free(C.a); free(F.a);
    return r;
}

int64_t or_mined_count(void *rp) { return ((or_mined *)rp)->len; }

/* i-th frequent pattern: n, rank labels[8], bits, results[4] (tau, mis, mni, frequent) */
void or_mined_get(void *rp, int64_t i, int32_t *n, int32_t *lab, uint32_t *bits, int64_t *res)
{
    or_mined *r = rp;
    *n = r->code[i].n;
    for (int j = 0; j < 8; j++) lab[j] = j < r->code[i].n ? r->code[i].lab[j] : 0;
    *bits = (uint32_t)r->code[i].bits;
    for (int j = 0; j < 4; j++) res[j] = r->res[4 * i + j];
}

void or_mined_levels(void *rp, int64_t *cand, int64_t *freq)
{
    or_mined *r = rp;
    for (int k = 0; k <= OR_MAXN; k++) { cand[k] = r->lvl_cand[k]; freq[k] = r->lvl_freq[k]; }
}

void or_mined_free(void *rp)
{
    or_mined *r = rp;
    if (!r) return;
    free(r->code); free(r->res); free(r);
}
