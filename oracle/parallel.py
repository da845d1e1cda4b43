"""Multi-process driver of the plain C oracle.

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU-baseline leg).  The
per-candidate work is the oracle's own single-threaded code (or_support, tier 1); this module
only spreads independent candidates over worker processes started with `spawn`, each holding its
own copy of the data graph.  `mine_parallel` is Algorithm 1 with each level's candidates
evaluated that way; it must return exactly what the oracle's own serial mining loop returns.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_G = None


def _init(labels, src, dst, seed, root_order):
    global _G
    import oracle
    _G = oracle.Graph(labels, src, dst, seed=seed, root_order=root_order)


def _eval(chunk):
    out = []
    for labels, edges, sigma, lam_num, mode, budget in chunk:
        r = _G.support(labels, edges, sigma=sigma, lam_num=lam_num, mode=mode, tier=1, budget=budget)
        out.append(None if r is None else (r["tau"], r["mis"], r["mni"], r["frequent"]))
    return out


class Pool:
    """`workers` spawned processes, each with the oracle graph of (labels, src, dst)."""

    def __init__(self, labels, src, dst, workers=None, seed=0x5EED, root_order="hash"):
        self.workers = workers or os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.workers, initializer=_init,
                             initargs=(np.asarray(labels, np.int32), np.asarray(src, np.int32),
                                       np.asarray(dst, np.int32), seed, root_order))

    def evaluate(self, items, mode="early", budget=0):
        """items: list of (labels, edges, sigma, lam_num); returns [(tau, mis, mni, frequent)], None
        for a pattern whose searches passed `budget` candidate vertices (budget > 0)."""
        if not items:
            return []
        k = max(1, min(256, len(items) // (4 * self.workers) + 1))
        chunks = [[(list(map(int, l)), [tuple(map(int, e)) for e in E], int(s), int(q), mode, int(budget))
                   for l, E, s, q in items[i:i + k]] for i in range(0, len(items), k)]
        out = []
        for part in self.pool.map(_eval, chunks):
            out.extend(part)
        return out

    def close(self):
        self.pool.close()
        self.pool.join()


def _edges_of(n, bits):
    edges, t = [], n * (n - 1) // 2 - 1
    for b in range(1, n):
        for a in range(b):
            if not (bits >> t) & 1:
                edges.append((a, b))
            t -= 1
    return edges


def mine_parallel(pool: Pool, labels, src, dst, sigma, lam_num, max_edges, lam_den=10**6):
    """Algorithm 1 over `pool`: level 2 = label pairs on data edges, each level's candidates
    evaluated in parallel (EARLY mode), next candidates by the oracle's predicate generator.
    Returns (patterns, levels) in the form of oracle.Graph.mine."""
    import oracle
    assert lam_den == 10**6
    labels = np.asarray(labels)
    og = oracle.Graph(labels, src, dst)
    present = sorted(set(int(x) for x in labels))
    rank = {l: og.rank(l) for l in present}
    label_of_rank = {r: l for l, r in rank.items()}
    pairs = set()
    for a, b in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if a != b:
            ra, rb = rank[int(labels[a])], rank[int(labels[b])]
            pairs.add((min(ra, rb), max(ra, rb)))
    C = sorted({(2,) + oracle.canonical([a, b], [(0, 1)])[:2] for a, b in pairs})
    found, levels = [], {}
    k = 2
    while C and k <= max_edges + 1 and k <= 8:
        items = []
        for n, labs, bits in C:
            items.append(([label_of_rank[r] for r in labs], _edges_of(n, bits), sigma, lam_num))
        res = pool.evaluate(items, mode="early_nomni")
        F = []
        for (n, labs, bits), (tau, mis, mni, freq) in zip(C, res):
            if freq:
                mni = max(tau, 1)  # mIS <= MNI: a frequent pattern's capped MNI is c
                F.append((n, labs, bits))
                found.append((n, tuple(labs), bits, tau, mis, mni))
        levels[k] = (len(C), len(F))
        if k + 1 <= max_edges + 1 and F:
            C = oracle.candidates([(list(labs), _edges_of(n, bits)) for n, labs, bits in F], max_edges)
        else:
            C = []
        k += 1
    found.sort(key=lambda p: (p[0], p[1], p[2]))
    return found, levels
