"""Seeded synthetic inputs shaped like the paper's workloads.

This module generates *inputs only*: data graphs (Erdos-Renyi, Chung-Lu power law), vertex
labels (uniform or Zipf) and query patterns (random trees, cycles, cliques, paths, stars).  It
holds none of the support-evaluation arithmetic, so both the CUDA path and the oracle can be fed
from it without sharing method code.

Random numbers come from one counter-based stream: the SplitMix64 generator of Steele, Lea and
Flood ("Fast splittable pseudorandom number generators", OOPSLA 2014), evaluated vectorised
(draw i of a stream seeded with s is mix(s + (i + 1) * 0x9E3779B97F4A7C15)).

The datasets of the paper (Gnutella, Epinions, Slashdot, wiki-Vote, MiCo; Table 1) and the
Citeseer / Patents / YouTube graphs the workloads are named after are not available; these
generators stand in for their shapes (vertex and edge counts, label counts and skew, power-law
degrees).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


class Stream:
    """Counter-based SplitMix64 stream.  `next(k)` returns the next k uint64 draws."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0

    def next(self, k: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + 1 + k, dtype=np.uint64)
        self.pos += k
        with np.errstate(over="ignore"):
            z = self.seed + idx * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _C1
            z = (z ^ (z >> np.uint64(27))) * _C2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int) -> np.ndarray:
        """k doubles in [0, 1) from the top 53 bits of each draw."""
        return (self.next(k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, k: int, n: int) -> np.ndarray:
        """k integers in [0, n) (floor of a uniform double times n)."""
        u = self.uniform(k)
        return np.minimum((u * n).astype(np.int64), n - 1)

    def permutation(self, n: int) -> np.ndarray:
        """Random permutation of range(n) (argsort of n draws, stable)."""
        return np.argsort(self.next(n), kind="stable").astype(np.int64)


def _distinct_edges(st: Stream, nv: int, ne: int, draw_pairs) -> tuple[np.ndarray, np.ndarray]:
    """Draw endpoint pairs until exactly `ne` distinct undirected non-loop edges exist.

    Edges are kept in order of their first draw, so the result is a deterministic function of
    the stream."""
    keys_all = np.empty(0, dtype=np.int64)
    need = ne
    while True:
        batch = int(need * 1.3) + 1024
        u, v = draw_pairs(batch)
        keep = u != v
        u, v = u[keep], v[keep]
        lo = np.minimum(u, v)
        hi = np.maximum(u, v)
        keys_all = np.concatenate([keys_all, lo * nv + hi])
        uniq, first = np.unique(keys_all, return_index=True)
        if uniq.size >= ne:
            order = np.sort(first)[:ne]
            keys = keys_all[order]
            return (keys // nv).astype(np.int32), (keys % nv).astype(np.int32)
        need = ne - uniq.size
        # keep only the first occurrences so the array does not grow without bound
        keys_all = keys_all[np.sort(first)]


def erdos_renyi(nv: int, ne: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Exactly `ne` distinct uniform random undirected edges on `nv` vertices."""
    st = Stream(seed)

    def draw(k):
        return st.integers(k, nv), st.integers(k, nv)

    return _distinct_edges(st, nv, ne, draw)


def chung_lu(nv: int, ne: int, gamma: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Chung-Lu power-law graph: vertex i has weight (i+1)^(-1/(gamma-1)); both endpoints of each
    drawn edge are i.i.d. proportional to weight (inverse-CDF sampling); self-loops and duplicates
    are rejected until exactly `ne` distinct edges exist.  Vertex ids are then randomly permuted so
    that id order carries no degree information."""
    st = Stream(seed)
    w = np.power(np.arange(1, nv + 1, dtype=np.float64), -1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]

    def draw(k):
        a = np.searchsorted(cdf, st.uniform(k), side="right")
        b = np.searchsorted(cdf, st.uniform(k), side="right")
        return np.minimum(a, nv - 1).astype(np.int64), np.minimum(b, nv - 1).astype(np.int64)

    src, dst = _distinct_edges(st, nv, ne, draw)
    perm = st.permutation(nv)
    return perm[src].astype(np.int32), perm[dst].astype(np.int32)


def labels_uniform(nv: int, nl: int, seed: int) -> np.ndarray:
    return Stream(seed).integers(nv, nl).astype(np.int32)


def labels_zipf(nv: int, nl: int, s: float, seed: int) -> np.ndarray:
    """i.i.d. labels with P(label = k-1) proportional to k^(-s), k = 1..nl."""
    p = np.power(np.arange(1, nl + 1, dtype=np.float64), -s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    u = Stream(seed).uniform(nv)
    return np.minimum(np.searchsorted(cdf, u, side="right"), nl - 1).astype(np.int32)


# ----------------------------------------------------------------------------- patterns

def _tree_prufer(n: int, st: Stream) -> list[tuple[int, int]]:
    if n == 2:
        return [(0, 1)]
    seq = [int(x) for x in st.integers(n - 2, n)]
    degree = [1] * n
    for x in seq:
        degree[x] += 1
    edges = []
    for x in seq:
        leaf = min(i for i in range(n) if degree[i] == 1)
        edges.append((leaf, x))
        degree[leaf] -= 1
        degree[x] -= 1
    u, v = [i for i in range(n) if degree[i] == 1]
    edges.append((u, v))
    return edges


def pattern_edges(shape: str, n: int, st: Stream) -> list[tuple[int, int]]:
    if shape == "tree":
        return _tree_prufer(n, st)
    if shape == "path":
        return [(i, i + 1) for i in range(n - 1)]
    if shape == "star":
        return [(0, i) for i in range(1, n)]
    if shape == "cycle":
        if n < 3:
            return [(0, 1)]
        return [(i, (i + 1) % n) for i in range(n)]
    if shape == "clique":
        return [(i, j) for i in range(n) for j in range(i + 1, n)]
    raise ValueError(shape)


def random_patterns(count: int, sizes, shapes, graph_labels: np.ndarray, seed: int):
    """`count` patterns; size uniform over `sizes`, shape uniform over `shapes`, each vertex label
    drawn from the data graph's label distribution (the label of a uniformly random data vertex),
    so that patterns are not trivially absent.  Returns a list of (labels int32[n], edges int32[m,2])."""
    st = Stream(seed)
    sizes = list(sizes)
    shapes = list(shapes)
    nv = graph_labels.shape[0]
    out = []
    for _ in range(count):
        n = sizes[int(st.integers(1, len(sizes))[0])]
        shape = shapes[int(st.integers(1, len(shapes))[0])]
        edges = pattern_edges(shape, n, st)
        lab = graph_labels[st.integers(n, nv)].astype(np.int32)
        out.append((lab, np.asarray(edges, dtype=np.int32).reshape(-1, 2)))
    return out


# ----------------------------------------------------------------------------- named workloads

# (name, graph kind, |V|, |E|, labels, label law, gamma)
GRAPHS = {
    "citeseer": dict(kind="er", nv=3312, ne=4732, nl=6, law="uniform", zipf_s=None, gamma=None, seed=1001),
    "mico": dict(kind="cl", nv=100_000, ne=1_080_000, nl=29, law="zipf", zipf_s=1.2, gamma=2.3, seed=1002),
    "cl1m": dict(kind="cl", nv=1_000_000, ne=10_000_000, nl=37, law="zipf", zipf_s=1.0, gamma=2.3, seed=1003),
    "patents": dict(kind="cl", nv=3_774_768, ne=16_518_947, nl=37, law="zipf", zipf_s=1.0, gamma=2.3, seed=1004),
    "youtube": dict(kind="cl", nv=4_600_000, ne=43_900_000, nl=80, law="zipf", zipf_s=1.0, gamma=2.3, seed=1005),
}


def make_graph(name: str = None, **kw):
    """Returns (labels int32[nv], src int32[ne], dst int32[ne]) for a named or custom graph."""
    spec = dict(GRAPHS[name]) if name is not None else {}
    spec.update(kw)
    nv, ne, nl, seed = spec["nv"], spec["ne"], spec["nl"], spec["seed"]
    if spec["kind"] == "er":
        src, dst = erdos_renyi(nv, ne, seed)
    else:
        src, dst = chung_lu(nv, ne, spec["gamma"], seed)
    if spec["law"] == "uniform":
        lab = labels_uniform(nv, nl, seed + 7919)
    else:
        lab = labels_zipf(nv, nl, spec["zipf_s"], seed + 7919)
    return lab, src, dst


def batch_level_patterns(graph_labels: np.ndarray, count: int = 2000, seed: int = 2003):
    """The batched-level workload: `count` patterns, n uniform in 3..7, shape uniform over
    {random tree, cycle, clique}, labels from the graph's label distribution."""
    return random_patterns(count, range(3, 8), ["tree", "cycle", "clique"], graph_labels, seed)
