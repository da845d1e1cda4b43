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
