"""Pure-Python brute force on tiny inputs, written from the paper's definitions only.

Used to pin the oracle: it never calls the oracle or the CUDA library.
  - maps: Sec. 2.1.4 (injective, label preserving, pattern edge -> data edge) and Sec. 2.4 (M).
  - independence: Sec. 2.4.1 (no two maps share a data vertex).
  - maximum independent set: Sec. 2.4.2; maximal: Sec. 2.4.3.
  - MNI: Sec. 2.4.4.
"""
from __future__ import annotations

import itertools


def adjacency(nv, edges):
    adj = [set() for _ in range(nv)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def maps(data_labels, data_edges, pat_labels, pat_edges):
    """All maps as tuples f with f[u] = image of pattern vertex u."""
    nv = len(data_labels)
    adj = adjacency(nv, data_edges)
    n = len(pat_labels)
    out = []
    for f in itertools.permutations(range(nv), n):
        if any(data_labels[f[u]] != pat_labels[u] for u in range(n)):
            continue
        if all(f[b] in adj[f[a]] for a, b in pat_edges):
            out.append(f)
    return out


def mni(M, n):
    if not M:
        return 0
    return min(len({f[u] for f in M}) for u in range(n))


def vertex_sets(M):
    return sorted({frozenset(f) for f in M}, key=sorted)


def maximum_is(M):
    """Size of a maximum independent set of maps (only vertex sets matter: maps with the same
    vertex set conflict with each other)."""
    sets = vertex_sets(M)
    best = 0

    def rec(i, used, k):
        nonlocal best
        if k + (len(sets) - i) <= best:
            return
        if i == len(sets):
            best = max(best, k)
            return
        if not (sets[i] & used):
            rec(i + 1, used | sets[i], k + 1)
        rec(i + 1, used, k)

    rec(0, frozenset(), 0)
    return best


def maximal_is_sizes(M):
    """Sizes of all maximal independent sets of maps (= every size a greedy order can give)."""
    sets = vertex_sets(M)
    sizes = set()
    for r in range(len(sets) + 1):
        for comb in itertools.combinations(range(len(sets)), r):
            chosen = [sets[i] for i in comb]
            used = set()
            ok = True
            for s in chosen:
                if s & used:
                    ok = False
                    break
                used |= s
            if not ok:
                continue
            if all(sets[j] & used for j in range(len(sets)) if j not in comb):
                sizes.add(r)
    return sizes


def is_independent(sel):
    used = set()
    for f in sel:
        if set(f) & used:
            return False
        used |= set(f)
    return True


def is_maximal(sel, M):
    used = set()
    for f in sel:
        used |= set(f)
    return all(set(f) & used for f in M)


# ----------------------------------------------------------------------------- mining, Algorithm 1
# A level-wise miner written from Algorithm 1 (Sec. 3.2) on top of the definitions above, used to
# pin the oracle's mining loop.  It follows the library's fixed readings where the paper leaves a
# choice open:
#   R1 labels are ranked by ascending frequency (ties by label id);
#   R2 canonical form = lexicographic minimum over all vertex orders of
#      (rank labels in order, then for j = 1..n-1 and i = 0..j-1 the bit "i is NOT adjacent to j");
#   R3 matching order: pi_0 = canonical vertex 0, then the smallest unvisited vertex adjacent to a
#      visited one;
#   R4 greedy order: maps sorted by (H(seed, root), root, e[pi_1], ..., e[pi_{n-1}]),
#      root = e[pi_0], H = one SplitMix64 step from state seed XOR root;
#   R5 EARLY counts: min(count, c) with c = max(tau, 1); frequent <=> mIS >= c.
# Candidates of the next level are the plain predicate of Algorithms 2-4: a connected k-vertex P
# is a candidate iff it is not a clique and two non-adjacent vertices u != v have P-u and P-v in
# F, or it is a clique and every P-u is in F.  Extensions try every label of the data graph.

_M64 = (1 << 64) - 1


def splitmix_step(seed, r):
    z = ((seed ^ r) + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def label_ranks(data_labels):
    cnt = {}
    for l in data_labels:
        cnt[l] = cnt.get(l, 0) + 1
    order = sorted(cnt, key=lambda l: (cnt[l], l))
    return {l: r for r, l in enumerate(order)}


def canon(labels, adj):
    """(code, order): code = (labels tuple, bits tuple) minimal over all vertex orders; order[p]
    = vertex at canonical position p.  adj is a set of frozenset pairs."""
    n = len(labels)
    best = None
    for perm in itertools.permutations(range(n)):
        code = (tuple(labels[v] for v in perm),
                tuple(0 if frozenset((perm[i], perm[j])) in adj else 1
                      for j in range(1, n) for i in range(j)))
        if best is None or code < best[0]:
            best = (code, perm)
    return best


def pattern_of_code(code):
    labels, bits = code
    n = len(labels)
    adj, t = set(), 0
    for j in range(1, n):
        for i in range(j):
            if not bits[t]:
                adj.add(frozenset((i, j)))
            t += 1
    return list(labels), adj


def connected_pattern(n, adj):
    seen, todo = {0}, [0]
    while todo:
        u = todo.pop()
        for v in range(n):
            if v not in seen and frozenset((u, v)) in adj:
                seen.add(v)
                todo.append(v)
    return len(seen) == n


def matching_order(n, adj):
    pi, seen = [0], {0}
    while len(pi) < n:
        nxt = min(v for v in range(n) if v not in seen and any(frozenset((u, v)) in adj for u in seen))
        pi.append(nxt)
        seen.add(nxt)
    return pi


def maps_backtrack(rank_of_vertex, nbrs, labels, adj):
    """All maps of the pattern (vertex u -> data vertex with rank label labels[u], injective,
    pattern edges on data edges), by plain backtracking in vertex order."""
    n = len(labels)
    nv = len(rank_of_vertex)
    out, cur = [], []

    def rec(u):
        if u == n:
            out.append(tuple(cur))
            return
        for d in range(nv):
            if rank_of_vertex[d] != labels[u] or d in cur:
                continue
            if all(cur[w] in nbrs[d] for w in range(u) if frozenset((w, u)) in adj):
                cur.append(d)
                rec(u + 1)
                cur.pop()

    rec(0)
    return out


def tau_exact(sigma, num, den, n):
    return sigma * ((n - 1) * num + den) // (n * den)


def evaluate_code(code, rank_of_vertex, nbrs, sigma, num, den, seed):
    """(tau, min(mIS, c), min(MNI, c), frequent) of a rank-space canonical pattern."""
    labels, adj = pattern_of_code(code)
    n = len(labels)
    M = maps_backtrack(rank_of_vertex, nbrs, labels, adj)
    pi = matching_order(n, adj)
    M.sort(key=lambda e: (splitmix_step(seed, e[pi[0]]), e[pi[0]]) + tuple(e[p] for p in pi[1:]))
    used, mis = set(), 0
    for e in M:
        if not (set(e) & used):
            used |= set(e)
            mis += 1
    t = tau_exact(sigma, num, den, n)
    c = max(t, 1)
    return t, min(mis, c), min(mni(M, n), c), mis >= c


def mine(data_labels, data_edges, sigma, num, den, max_edges, seed=0x5EED):
    """Algorithm 1: returns (patterns, levels); patterns = sorted list of (n, rank labels, bits
    as an integer with the first bit most significant, tau, mis, mni) of the frequent patterns,
    levels = {k: (candidates, frequent)}."""
    ranks = label_ranks(data_labels)
    rv = [ranks[l] for l in data_labels]
    nbrs = adjacency(len(data_labels), data_edges)
    all_ranks = sorted(set(rv))
    # level 2: one candidate per label pair found on a data edge
    C = set()
    for a, b in data_edges:
        if a != b:
            C.add(canon([rv[a], rv[b]], {frozenset((0, 1))})[0])
    found, levels = [], {}
    k = 2
    while C and k <= max_edges + 1 and k <= 8:
        F = set()
        for code in C:
            t, mis_c, mni_c, freq = evaluate_code(code, rv, nbrs, sigma, num, den, seed)
            if freq:
                F.add(code)
                bits = 0
                for x in code[1]:
                    bits = (bits << 1) | x
                found.append((k, code[0], bits, t, mis_c, mni_c))
        levels[k] = (len(C), len(F))
        # candidates of level k+1 from F (never from C)
        C = set()
        if k + 1 <= max_edges + 1:
            for code in F:
                base_lab, base_adj = pattern_of_code(code)
                for lab_new in all_ranks:
                    for S in range(1, 1 << k):
                        adj = set(base_adj) | {frozenset((i, k)) for i in range(k) if S >> i & 1}
                        if len(adj) > max_edges:
                            continue
                        labs = base_lab + [lab_new]
                        if is_candidate(labs, adj, F):
                            C.add(canon(labs, adj)[0])
        k += 1
    found.sort(key=lambda p: (p[0], p[1], p[2]))
    return found, levels


def minus_vertex(labels, adj, u):
    keep = [v for v in range(len(labels)) if v != u]
    idx = {v: i for i, v in enumerate(keep)}
    sub = {frozenset((idx[a], idx[b])) for a, b in (tuple(e) for e in adj) if a != u and b != u}
    return [labels[v] for v in keep], sub


def is_candidate(labels, adj, F):
    n = len(labels)

    def in_F(u):
        sl, sa = minus_vertex(labels, adj, u)
        return connected_pattern(n - 1, sa) and canon(sl, sa)[0] in F

    if len(adj) == n * (n - 1) // 2:
        return all(in_F(u) for u in range(n))
    inF = [in_F(u) for u in range(n)]
    return any(inF[u] and inF[v] for u in range(n) for v in range(u + 1, n)
               if frozenset((u, v)) not in adj)


# ----------------------------------------------------------------------------- edge labels
# Sec. 2.3.5: an edge (u, v) with label l is replaced by edges (u, w), (w, v) through a new vertex
# w labelled l.  extend_graph / extend_pattern write that transform out; maps_edge_labelled is
# the direct definition (injective, vertex labels kept, every pattern edge on a data edge with
# the same edge label) that the transform must reproduce.

def extend_graph(labels, edges, edge_labels):
    """Extended graph: (labels, edges) with one vertex per kept edge; edge label l becomes label
    base + l, base = 1 + the largest vertex label.  Self-loops dropped; of repeated vertex pairs
    the first edge is kept."""
    base = max(labels) + 1 if len(labels) else 0
    lab = list(labels)
    out, seen = [], set()
    for (a, b), l in zip(edges, edge_labels):
        if a == b or frozenset((a, b)) in seen:
            continue
        seen.add(frozenset((a, b)))
        w = len(lab)
        lab.append(base + l)
        out += [(a, w), (w, b)]
    return lab, out, base


def extend_pattern(labels, edges, edge_labels, base):
    lab = list(labels)
    out = []
    for (a, b), l in zip(edges, edge_labels):
        w = len(lab)
        lab.append(base + l)
        out += [(a, w), (w, b)]
    return lab, out


def maps_edge_labelled(labels, edges, edge_labels, pat_labels, pat_edges, pat_edge_labels):
    elab = {}
    for (a, b), l in zip(edges, edge_labels):
        if a != b and frozenset((a, b)) not in elab:
            elab[frozenset((a, b))] = l
    n = len(pat_labels)
    out = []
    for f in itertools.permutations(range(len(labels)), n):
        if any(labels[f[u]] != pat_labels[u] for u in range(n)):
            continue
        if all(elab.get(frozenset((f[a], f[b]))) == l for (a, b), l in zip(pat_edges, pat_edge_labels)):
            out.append(f)
    return out


# ----------------------------------------------------------------------------- directed graphs
# Sec. 2.2 states the problem on directed graphs: a map keeps labels, is injective, and sends
# every pattern arc a -> b to a data arc f(a) -> f(b).

def maps_directed(data_labels, data_arcs, pat_labels, pat_arcs):
    out_nb = [set() for _ in data_labels]
    for a, b in data_arcs:
        if a != b:
            out_nb[a].add(b)
    n = len(pat_labels)
    res = []
    for f in itertools.permutations(range(len(data_labels)), n):
        if any(data_labels[f[u]] != pat_labels[u] for u in range(n)):
            continue
        if all(f[b] in out_nb[f[a]] for a, b in pat_arcs):
            res.append(f)
    return res
