"""Pins of the oracle (CPU only).

Each test ties the oracle to something other than itself: values the paper prints for its worked
examples (tests/golden/), a pure-Python brute force written from the definitions
(tests/bruteforce.py), Theorem 1's bounds, networkx graph isomorphism, and the agreement of the
oracle's two independent tiers (brute force over V^n with an explicit sorted map list, and
per-root backtracking)."""
from __future__ import annotations

import json
import os
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest

import oracle
from tests import bruteforce as bf
from workloads import Stream, erdos_renyi, labels_uniform, pattern_edges

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def graph_of(d, seed=oracle.Graph.DEFAULT_SEED):
    e = np.asarray(d["data_edges"], dtype=np.int32)
    return oracle.Graph(d["data_labels"], e[:, 0], e[:, 1], seed=seed)


# ----------------------------------------------------------------------------- tau (Eq. tau)

def test_tau_paper_examples():
    d = load("running_example.json")
    for ex in d["tau_examples"]:
        assert oracle.tau(ex["sigma"], ex["lambda"], ex["n"]) == ex["tau"], ex["cite"]


@pytest.mark.parametrize("sigma", [1, 2, 3, 7, 300, 1000, 20000, 10**12])
@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_tau_endpoints(sigma, n):
    # Sec. 3.1.1: lambda = 1 gives tau = sigma; lambda = 0 gives sigma / n (floored)
    assert oracle.tau(sigma, 1.0, n) == sigma
    assert oracle.tau(sigma, 0.0, n) == sigma // n


def test_tau_monotone_and_exact_rounding():
    # tau is non-decreasing in lambda and lies between the two endpoints
    for sigma in (3, 10, 299, 1000):
        for n in range(2, 9):
            prev = -1
            for p in range(0, 1_000_001, 50_000):
                t = oracle.tau_q(sigma, p, 1_000_000, n)
                assert sigma // n <= t <= sigma
                assert t >= prev
                prev = t
    # a case where evaluating the formula in doubles rounds the other way: sigma = 3, n = 6,
    # lambda = 0.6 -> exactly 3 * 0.5 + 0.5 = 2.0
    assert oracle.tau(3, 0.6, 6) == 2
    assert Fraction(3) * (1 - Fraction(1, 6)) * Fraction(6, 10) + Fraction(3, 6) == 2


def test_tau_config_table():
    # sigma = 300, lambda = 0.5 for n = 2..6
    assert [oracle.tau(300, 0.5, n) for n in range(2, 7)] == [225, 200, 187, 180, 175]


# ----------------------------------------------------------------------------- hash (reading R4)

def test_hash_is_splitmix64():
    # Published SplitMix64 test vector: state 1234567 -> first output 6457827717110365317
    assert oracle.hash64(1234567, 0) == 6457827717110365317
    # the stream in workloads/ is the same generator
    assert int(Stream(1234567).next(1)[0]) == 6457827717110365317


# ----------------------------------------------------------------------------- running example

def test_running_example_maps_match_paper():
    d = load("running_example.json")
    P = d["P1"]
    M = bf.maps(d["data_labels"], d["data_edges"], P["labels"], P["edges"])
    assert sorted(M) == sorted(tuple(x) for x in d["P1_maps_u1u2u3"])
    g = graph_of(d)
    r0 = g.support(P["labels"], P["edges"], sigma=2, lam=1.0, mode="full", tier=0)
    assert r0["n_maps"] == 6
    assert g.count_maps(P["labels"], P["edges"]) == 6


def test_running_example_P1_metrics():
    d = load("running_example.json")
    P = d["P1"]
    M = bf.maps(d["data_labels"], d["data_edges"], P["labels"], P["edges"])
    assert bf.mni(M, 3) == d["P1_MNI"]
    assert bf.maximum_is(M) == d["P1_MIS"]
    assert bf.maximal_is_sizes(M) == set(d["P1_mIS_possible"])
    seen = set()
    for seed in range(64):
        g = graph_of(d, seed=seed)
        for tier in (0, 1):
            r = g.support(P["labels"], P["edges"], sigma=2, lam=1.0, mode="full", tier=tier,
                          want_selected=True)
            assert r["mni"] == d["P1_MNI"]
            assert r["mis"] in d["P1_mIS_possible"]
            sets = {frozenset(f) for f in M}
            assert all(frozenset(s) in sets for s in r["selected"])
            assert bf.is_independent(r["selected"]) and bf.is_maximal(r["selected"], M)
            seen.add(r["mis"])
            # frequent <=> mIS >= tau (sigma = 2, lambda = 1 -> tau = 2), Sec. 3.1.1
            assert r["tau"] == 2 and r["frequent"] == (r["mis"] >= 2)
    assert seen == {1, 2}  # both maximal sets of Sec. 3.1.1 are reached by some seed


def test_running_example_P1_early_tau1():
    # Sec. 3.1.1: sigma = 2, lambda = 0.25 -> tau = 1; FLEXIS stops at the first match and
    # declares P1 frequent
    d = load("running_example.json")
    g = graph_of(d)
    for tier in (0, 1):
        r = g.support(d["P1"]["labels"], d["P1"]["edges"], sigma=2, lam=0.25, mode="early", tier=tier)
        assert r["tau"] == 1 and r["mis"] == 1 and r["frequent"]
        # sigma = 3, lambda = 1: P1 infrequent under mIS (but MNI = 3 would call it frequent)
        r = g.support(d["P1"]["labels"], d["P1"]["edges"], sigma=3, lam=1.0, mode="full", tier=tier)
        assert r["tau"] == 3 and not r["frequent"] and r["mni"] == 3


def test_running_example_P2():
    d = load("running_example.json")
    P = d["P2"]
    M = bf.maps(d["data_labels"], d["data_edges"], P["labels"], P["edges"])
    assert len(M) == d["P2_maps"]
    assert bf.mni(M, 3) == d["P2_MNI"] and bf.maximum_is(M) == d["P2_MIS"]
    g = graph_of(d)
    for tier in (0, 1):
        r = g.support(P["labels"], P["edges"], sigma=1, lam=1.0, mode="full", tier=tier)
        assert r["mis"] == d["P2_MIS"] and r["mni"] == d["P2_MNI"]


# ----------------------------------------------------------------------------- Theorem 1 example

def test_malvisual_theorem1_example():
    d = load("malvisual.json")
    P = d["P"]
    M = bf.maps(d["data_labels"], d["data_edges"], P["labels"], P["edges"])
    assert len(M) == d["maps"] and bf.mni(M, 4) == d["MNI"]
    assert bf.maximum_is(M) == d["MIS"]
    sizes = bf.maximal_is_sizes(M)
    assert sizes == set(d["mIS_possible_bruteforce"]) and set(d["mIS_printed"]) <= sizes
    seen = set()
    for seed in range(200):
        g = graph_of(d, seed=seed)
        r0 = g.support(P["labels"], P["edges"], sigma=1, lam=1.0, mode="full", tier=0, want_selected=True)
        r1 = g.support(P["labels"], P["edges"], sigma=1, lam=1.0, mode="full", tier=1, want_selected=True)
        assert r0["n_maps"] == 48 and r0["mni"] == r1["mni"] == 5
        assert r0["mis"] == r1["mis"] and r0["selected"] == r1["selected"]
        assert bf.is_independent(r1["selected"]) and bf.is_maximal(r1["selected"], M)
        # Theorem 1: m <= MIS <= m * n
        assert r1["mis"] <= d["MIS"] <= 4 * r1["mis"]
        seen.add(r1["mis"])
    assert seen <= sizes and 4 in seen


# ----------------------------------------------------------------------------- random tiny graphs

def tiny_cases(count, seed):
    st = Stream(seed)
    out = []
    shapes = ["path", "star", "cycle", "clique", "tree"]
    for _ in range(count):
        nv = 5 + int(st.integers(1, 5)[0])           # 5..9 vertices
        ne = min(nv * (nv - 1) // 2, nv + int(st.integers(1, nv + 3)[0]))
        nl = 1 + int(st.integers(1, 3)[0])            # 1..3 labels
        s = int(st.next(1)[0] % (1 << 31))
        src, dst = erdos_renyi(nv, ne, s)
        lab = labels_uniform(nv, nl, s + 1)
        n = 2 + int(st.integers(1, 3)[0])             # 2..4 pattern vertices
        shape = shapes[int(st.integers(1, len(shapes))[0])]
        pe = pattern_edges(shape, n, st)
        pl = [int(x) for x in st.integers(n, nl)]
        out.append((lab, src, dst, pl, pe, s))
    return out


def test_tiers_agree_and_invariants():
    for lab, src, dst, pl, pe, s in tiny_cases(120, 17):
        edges = list(zip(src.tolist(), dst.tolist()))
        M = bf.maps(lab.tolist(), edges, pl, pe)
        n = len(pl)
        g = oracle.Graph(lab, src, dst, seed=s)
        for sigma, lam in ((1, 1.0), (3, 0.5), (5, 0.0)):
            r0 = g.support(pl, pe, sigma=sigma, lam=lam, mode="full", tier=0, want_selected=True)
            r1 = g.support(pl, pe, sigma=sigma, lam=lam, mode="full", tier=1, want_selected=True)
            e0 = g.support(pl, pe, sigma=sigma, lam=lam, mode="early", tier=0)
            e1 = g.support(pl, pe, sigma=sigma, lam=lam, mode="early", tier=1)
            assert r0["n_maps"] == len(M) == g.count_maps(pl, pe)
            assert (r0["mis"], r0["mni"]) == (r1["mis"], r1["mni"])
            assert r0["selected"] == r1["selected"]
            assert r0["mni"] == bf.mni(M, n)
            assert bf.is_independent(r1["selected"]) and bf.is_maximal(r1["selected"], M)
            # mIS <= MNI (m disjoint maps give each pattern vertex m distinct images)
            assert r1["mis"] <= r1["mni"]
            cap = max(r0["tau"], 1)
            assert e0["mis"] == e1["mis"] == min(r0["mis"], cap)
            assert e0["mni"] == e1["mni"] == min(r0["mni"], cap)
            assert e0["frequent"] == e1["frequent"] == r0["frequent"] == (r0["mis"] >= cap)
        if len(bf.vertex_sets(M)) <= 40:
            big = bf.maximum_is(M)
            # Theorem 1: m <= MIS <= m n
            assert r1["mis"] <= big <= n * r1["mis"]


def test_relabelling_invariance():
    # the result depends on the pattern only up to isomorphism
    st = Stream(99)
    for lab, src, dst, pl, pe, s in tiny_cases(40, 5):
        g = oracle.Graph(lab, src, dst, seed=s)
        n = len(pl)
        perm = [int(x) for x in st.permutation(n)]
        pl2 = [0] * n
        for u in range(n):
            pl2[perm[u]] = pl[u]
        pe2 = [(perm[a], perm[b]) for a, b in pe]
        a = g.support(pl, pe, sigma=2, lam=0.5, mode="full", tier=1, want_selected=True)
        b = g.support(pl2, pe2, sigma=2, lam=0.5, mode="full", tier=1, want_selected=True)
        assert (a["mis"], a["mni"], a["selected"]) == (b["mis"], b["mni"], b["selected"])


def greedy_matching(lab, src, dst, la, lb, seed):
    """Textbook greedy maximal matching of the a-b label edges, edges taken in the order
    (H(seed, a-endpoint), a-endpoint, b-endpoint), H = SplitMix64 step from state seed ^ a."""
    M64 = (1 << 64) - 1

    def H(r):
        z = ((seed ^ r) + 0x9E3779B97F4A7C15) & M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    E = set()
    for u, v in zip(src.tolist(), dst.tolist()):
        if u == v:
            continue
        for x, y in ((u, v), (v, u)):
            if lab[x] == la and lab[y] == lb:
                E.add((x, y))
    used = set()
    k = 0
    for x, y in sorted(E, key=lambda e: (H(e[0]), e[0], e[1])):
        if x not in used and y not in used:
            used |= {x, y}
            k += 1
    return k


def test_two_vertex_pattern_is_greedy_matching():
    for idx, (lab, src, dst, _, _, s) in enumerate(tiny_cases(60, 31)):
        if len(set(lab.tolist())) < 2:
            continue
        g = oracle.Graph(lab, src, dst, seed=s)
        a, b = sorted(set(lab.tolist()))[:2]
        # the root is the rarer label (ties: smaller id), reading R1 + R2
        ca, cb = int((lab == a).sum()), int((lab == b).sum())
        ra, rb = (a, b) if (ca, a) < (cb, b) else (b, a)
        want = greedy_matching(lab, src, dst, ra, rb, s)
        for tier in (0, 1):
            r = g.support([a, b], [(0, 1)], sigma=1, lam=1.0, mode="full", tier=tier)
            assert r["mis"] == want


# ------------------------------------------------------------------ root-order variant: vertex id

def greedy_matching_by_id(lab, src, dst, la, lb):
    """Textbook greedy maximal matching of the a-b label edges taken in lexicographic order of
    (a-endpoint, b-endpoint)."""
    E = sorted({(x, y) for u, v in zip(src.tolist(), dst.tolist()) if u != v
                for x, y in ((u, v), (v, u)) if lab[x] == la and lab[y] == lb})
    used, k = set(), 0
    for x, y in E:
        if x not in used and y not in used:
            used |= {x, y}
            k += 1
    return k


def test_id_root_order_tiers_agree_and_invariants():
    differs = 0
    for lab, src, dst, pl, pe, s in tiny_cases(120, 23):
        edges = list(zip(src.tolist(), dst.tolist()))
        M = bf.maps(lab.tolist(), edges, pl, pe)
        g = oracle.Graph(lab, src, dst, seed=s, root_order="id")
        gh = oracle.Graph(lab, src, dst, seed=s)
        r0 = g.support(pl, pe, sigma=1, lam=1.0, mode="full", tier=0, want_selected=True)
        r1 = g.support(pl, pe, sigma=1, lam=1.0, mode="full", tier=1, want_selected=True)
        assert (r0["mis"], r0["mni"], r0["selected"]) == (r1["mis"], r1["mni"], r1["selected"])
        assert bf.is_independent(r1["selected"]) and bf.is_maximal(r1["selected"], M)
        assert r1["mis"] <= r1["mni"] == bf.mni(M, len(pl))
        # the seed plays no part in id order
        g2 = oracle.Graph(lab, src, dst, seed=s + 12345, root_order="id")
        assert g2.support(pl, pe, sigma=1, lam=1.0, mode="full", tier=1, want_selected=True)["selected"] == r1["selected"]
        differs += gh.support(pl, pe, sigma=1, lam=1.0, mode="full", tier=1, want_selected=True)["selected"] != r1["selected"]
    assert differs > 0  # the two orders are really different orders


def test_id_root_order_two_vertex_pattern_is_lexicographic_greedy_matching():
    for lab, src, dst, _, _, s in tiny_cases(60, 37):
        if len(set(lab.tolist())) < 2:
            continue
        g = oracle.Graph(lab, src, dst, seed=s, root_order="id")
        a, b = sorted(set(lab.tolist()))[:2]
        ca, cb = int((lab == a).sum()), int((lab == b).sum())
        ra, rb = (a, b) if (ca, a) < (cb, b) else (b, a)
        want = greedy_matching_by_id(lab, src, dst, ra, rb)
        for tier in (0, 1):
            assert g.support([a, b], [(0, 1)], sigma=1, lam=1.0, mode="full", tier=tier)["mis"] == want


def test_id_root_order_path_closed_form():
    # a one-label path 0-1-...-(k-1): in id order root 0 takes edge (0,1), root 2 takes (2,3), ...
    for k in (2, 3, 7, 10, 31):
        lab = np.zeros(k, np.int32)
        src = np.arange(k - 1, dtype=np.int32)
        g = oracle.Graph(lab, src, src + 1, root_order="id")
        r = g.support([0, 0], [(0, 1)], sigma=1, lam=1.0, mode="full", tier=1, want_selected=True)
        assert r["mis"] == k // 2
        assert sorted(tuple(sorted(m)) for m in r["selected"]) == [(2 * i, 2 * i + 1) for i in range(k // 2)]


# ----------------------------------------------------------------------------- canonical code

def nxg(labels, edges):
    G = nx.Graph()
    for i, l in enumerate(labels):
        G.add_node(i, l=l)
    G.add_edges_from(edges)
    return G


def test_canonical_code_vs_networkx_isomorphism():
    st = Stream(7)
    pats = []
    for _ in range(160):
        n = 2 + int(st.integers(1, 5)[0])
        pe = [(i, j) for i in range(n) for j in range(i + 1, n) if st.uniform(1)[0] < 0.5]
        pl = [int(x) for x in st.integers(n, 2)]
        pats.append((pl, pe))
    codes = [oracle.canonical(pl, pe)[:2] for pl, pe in pats]
    nm = lambda a, b: a["l"] == b["l"]
    for i in range(len(pats)):
        # invariance under relabelling
        n = len(pats[i][0])
        perm = [int(x) for x in st.permutation(n)]
        pl2 = [0] * n
        for u in range(n):
            pl2[perm[u]] = pats[i][0][u]
        pe2 = [(perm[a], perm[b]) for a, b in pats[i][1]]
        assert oracle.canonical(pl2, pe2)[:2] == codes[i]
        for j in range(i + 1, min(len(pats), i + 25)):
            if len(pats[i][0]) != len(pats[j][0]):
                continue
            iso = nx.is_isomorphic(nxg(*pats[i]), nxg(*pats[j]), node_match=nm)
            assert (codes[i] == codes[j]) == iso


def test_canonical_labels_sorted_and_perm_valid():
    labs, bits, perm = oracle.canonical([2, 0, 1, 0], [(0, 1), (1, 2), (2, 3)])
    assert list(labs) == sorted(labs) and sorted(perm) == [0, 1, 2, 3]


# ----------------------------------------------------------------------------- candidate generation

R, B, G_, Y = 0, 1, 2, 3
TRI = [(0, 1), (1, 2), (0, 2)]


def test_candidates_from_P1_P2():
    # Sec. 3.2.1, Fig. merge process: F_3 = {P1, P2} over labels {R, B}.  The 4-vertex
    # candidates are the five labelled diamonds and the K4 RRBB (derived by hand from the
    # predicate; the paper draws three of them).
    c = oracle.candidates([([R, B, R], TRI), ([B, B, R], TRI)])
    assert len(c) == 6
    K4 = oracle.canonical([R, R, B, B], [(i, j) for i in range(4) for j in range(i + 1, 4)])[:2]
    assert (4, *K4) in [(n, l, b) for n, l, b in c]
    diamonds = [
        ([R, R, B, B], [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3)]),  # spine RR, tips BB
        ([R, B, R, R], [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3)]),  # spine RB, tips RR
        ([R, B, R, B], [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3)]),  # spine RB, tips RB
        ([R, B, B, B], [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3)]),  # spine RB, tips BB
        ([B, B, R, R], [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3)]),  # spine BB, tips RR
    ]
    got = {(l, b) for n, l, b in c}
    for pl, pe in diamonds:
        assert oracle.canonical(pl, pe)[:2] in got


def test_candidates_automorphism_merge():
    # Sec. 3.2.1 Example 2 (Fig. trailed triangle): P = triangle (B, R, R) with a red tail on a
    # red vertex.  Merging its core graph with itself must give both "two tails on u2" and
    # "tails on u2 and u3".
    P = ([B, R, R, R], [(0, 1), (1, 2), (0, 2), (1, 3)])
    c = {(l, b) for n, l, b in oracle.candidates([P])}
    two_on_u2 = oracle.canonical([B, R, R, R, R], [(0, 1), (1, 2), (0, 2), (1, 3), (1, 4)])[:2]
    on_u2_u3 = oracle.canonical([B, R, R, R, R], [(0, 1), (1, 2), (0, 2), (1, 3), (2, 4)])[:2]
    assert two_on_u2 in c and on_u2_u3 in c


def test_candidates_clique():
    # Sec. 3.2.1 Fig. merging clique: triangles RGB, RGY, RBY, GBY give the K4 RGBY; without
    # GBY the post-check removes it.
    K4 = oracle.canonical([R, G_, B, Y], [(i, j) for i in range(4) for j in range(i + 1, 4)])[:2]
    F = [([R, G_, B], TRI), ([R, G_, Y], TRI), ([R, B, Y], TRI), ([G_, B, Y], TRI)]
    assert K4 in {(l, b) for n, l, b in oracle.candidates(F)}
    assert K4 not in {(l, b) for n, l, b in oracle.candidates(F[:3])}


def test_candidates_complete_by_brute_force():
    # every connected k-vertex pattern over the labels whose non-clique / clique predicate holds
    # is generated, and nothing else: compare with an exhaustive enumeration of labelled graphs
    import itertools
    st = Stream(3)
    for trial in range(6):
        labels = [0, 1]
        k = 3 + (trial % 2)
        # random set F of connected (k-1)-vertex patterns
        allp = []
        for lab in itertools.product(labels, repeat=k - 1):
            pairs = [(i, j) for i in range(k - 1) for j in range(i + 1, k - 1)]
            for mask in range(1, 1 << len(pairs)):
                e = [pairs[t] for t in range(len(pairs)) if mask >> t & 1]
                if nx.is_connected(nx.Graph(e)) and len({x for p in e for x in p}) == k - 1:
                    allp.append((list(lab), e))
        F = [p for p in allp if st.uniform(1)[0] < 0.5]
        if not F:
            continue
        Fc = {oracle.canonical(*p)[:2] for p in F}
        want = set()
        for lab in itertools.product(labels, repeat=k):
            pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
            for mask in range(1, 1 << len(pairs)):
                e = [pairs[t] for t in range(len(pairs)) if mask >> t & 1]
                Gx = nx.Graph()
                Gx.add_nodes_from(range(k))
                Gx.add_edges_from(e)
                if not nx.is_connected(Gx):
                    continue

                def sub_in(u):
                    H = Gx.copy()
                    H.remove_node(u)
                    if not nx.is_connected(H):
                        return False
                    idx = {v: i for i, v in enumerate(sorted(H.nodes))}
                    return oracle.canonical([lab[v] for v in sorted(H.nodes)],
                                            [(idx[a], idx[b]) for a, b in H.edges])[:2] in Fc

                clique = len(e) == k * (k - 1) // 2
                ins = [sub_in(u) for u in range(k)]
                if clique:
                    ok = all(ins)
                else:
                    ok = any(ins[u] and ins[v] and not Gx.has_edge(u, v)
                             for u in range(k) for v in range(u + 1, k))
                if ok:
                    want.add(oracle.canonical(list(lab), e)[:2])
        got = {(l, b) for n, l, b in oracle.candidates(F)}
        assert got == want


# ----------------------------------------------------------------------------- mining

def test_size_pruning_example():
    # Sec. 3.1.1: |V| = 40 and tau = 10 -> no frequent pattern has more than 4 vertices
    src, dst = erdos_renyi(40, 150, 4)
    lab = np.zeros(40, np.int32)
    g = oracle.Graph(lab, src, dst)
    pats, levels = g.mine(sigma=10, lam=1.0, max_edges=6)
    assert pats and max(p[0] for p in pats) <= 4


def test_mining_levels_consistent():
    src, dst = erdos_renyi(60, 150, 11)
    lab = labels_uniform(60, 2, 12)
    g = oracle.Graph(lab, src, dst)
    pats, levels = g.mine(sigma=4, lam=0.5, max_edges=3)
    # every reported pattern is frequent under its own evaluation and ordered by (n, code)
    keys = [(p[0], p[1], p[2]) for p in pats]
    assert keys == sorted(keys)
    for n, labs, bits, tau, mis, mni in pats:
        assert mis >= max(tau, 1) and mni >= mis
    for k, (cand, freq) in levels.items():
        assert freq == sum(1 for p in pats if p[0] == k) and freq <= cand


def mining_cases(count, seed):
    st = Stream(seed)
    out = []
    for _ in range(count):
        nv = 8 + int(st.integers(1, 5)[0])             # 8..12 vertices
        ne = nv + int(st.integers(1, nv)[0])           # nv .. 2nv - 1 edges
        nl = 1 + int(st.integers(1, 3)[0])             # 1..3 labels
        s = int(st.next(1)[0] % (1 << 31))
        src, dst = erdos_renyi(nv, ne, s)
        lab = labels_uniform(nv, nl, s + 1)
        sigma = 1 + int(st.integers(1, 4)[0])          # 1..4
        lam = (0.0, 0.5, 1.0)[int(st.integers(1, 3)[0])]
        max_edges = 2 + int(st.integers(1, 3)[0])      # 2..4
        out.append((lab, src, dst, sigma, lam, max_edges, s))
    return out


def test_mining_matches_python_level_wise_miner():
    # Algorithm 1 restated in plain Python over brute-force maps (tests/bruteforce.py): the
    # whole frequent set (codes, tau, mis, mni) and the per-level candidate and frequent counts
    # must be identical.  Seeds vary the greedy order; levels with infrequent candidates make
    # generating from C_k instead of F_k visible, and every level-2 label pair matters.
    saw_infrequent = 0
    for lab, src, dst, sigma, lam, max_edges, s in mining_cases(30, 2024):
        E = list(zip(src.tolist(), dst.tolist()))
        want, wlev = bf.mine(lab.tolist(), E, sigma, int(round(lam * 10**6)), 10**6, max_edges, seed=s)
        g = oracle.Graph(lab, src, dst, seed=s)
        got, glev = g.mine(sigma=sigma, lam=lam, max_edges=max_edges)
        assert glev == wlev, (sigma, lam, max_edges, glev, wlev)
        assert got == want, (sigma, lam, max_edges)
        saw_infrequent += sum(1 for c, f in wlev.values() if f < c)
    assert saw_infrequent >= 10


# ----------------------------------------------------------------------------- overlap graph, MIS

def test_maximum_independent_set_paper_examples():
    # Sec. 2.4.2: the MIS of P1 in D has 2 maps; the Theorem 1 example (Fig. malVisual) has MIS 4
    d = load("running_example.json")
    g = graph_of(d)
    assert g.max_independent_set(d["P1"]["labels"], d["P1"]["edges"]) == d["P1_MIS"] == 2
    assert g.max_independent_set(d["P2"]["labels"], d["P2"]["edges"]) == d["P2_MIS"] == 1
    inst, edges = g.overlap_graph(d["P1"]["labels"], d["P1"]["edges"])
    # the six maps of P1 form three instances {d1,d2,d5}, {d2,d3,d6}, {d3,d4,d7} in a path
    assert inst == [(0, 1, 4), (1, 2, 5), (2, 3, 6)] and edges == [(0, 1), (1, 2)]
    m = load("malvisual.json")
    gm = graph_of(m)
    assert gm.max_independent_set(m["P"]["labels"], m["P"]["edges"]) == m["MIS"] == 4


def test_overlap_graph_and_mis_match_brute_force():
    for lab, src, dst, pl, pe, s in tiny_cases(120, 23):
        edges = list(zip(src.tolist(), dst.tolist()))
        M = bf.maps(lab.tolist(), edges, pl, pe)
        g = oracle.Graph(lab, src, dst, seed=s)
        sets = bf.vertex_sets(M)
        got = g.overlap_graph(pl, pe)
        assert got is not None
        inst, cedges = got
        assert inst == sorted(tuple(sorted(x)) for x in sets)
        want_edges = [(a, b) for a in range(len(inst)) for b in range(a + 1, len(inst))
                      if set(inst[a]) & set(inst[b])]
        assert cedges == want_edges
        if len(sets) <= 40:
            big = g.max_independent_set(pl, pe, max_inst=40)
            assert big == bf.maximum_is(M)
            r = g.support(pl, pe, sigma=1, lam=1.0, mode="full", tier=1)
            # Theorem 1: mIS <= MIS <= n mIS
            assert r["mis"] <= big <= len(pl) * r["mis"]


# ----------------------------------------------------------------------------- edge labels

def edge_labelled_cases(count, seed):
    st = Stream(seed)
    out = []
    shapes = ["path", "star", "cycle", "tree"]
    for _ in range(count):
        nv = 5 + int(st.integers(1, 4)[0])
        ne = min(nv * (nv - 1) // 2, nv + int(st.integers(1, nv)[0]))
        s = int(st.next(1)[0] % (1 << 31))
        src, dst = erdos_renyi(nv, ne, s)
        lab = labels_uniform(nv, 2, s + 1)
        el = [int(x) for x in st.integers(ne, 2)]
        n = 2 + int(st.integers(1, 2)[0])              # 2..3 vertices, n + m <= 8
        pe = pattern_edges(shapes[int(st.integers(1, len(shapes))[0])], n, st)
        pl = [int(x) for x in st.integers(n, 2)]
        pel = [int(x) for x in st.integers(len(pe), 2)]
        out.append((lab, src, dst, el, pl, pe, pel, s))
    return out


def test_edge_label_extension_preserves_maps():
    # the maps of the extended pattern in the extended graph are the edge-label-respecting maps
    # of the original pattern (one extended map per original map: the graph is simple)
    for lab, src, dst, el, pl, pe, pel, s in edge_labelled_cases(80, 31):
        E = list(zip(src.tolist(), dst.tolist()))
        want = bf.maps_edge_labelled(lab.tolist(), E, el, pl, pe, pel)
        xl, xe, base = bf.extend_graph(lab.tolist(), E, el)
        pxl, pxe = bf.extend_pattern(pl, pe, pel, base)
        g = oracle.Graph(np.asarray(xl, np.int32), np.asarray([a for a, b in xe], np.int32),
                         np.asarray([b for a, b in xe], np.int32), seed=s)
        r = g.support(pxl, pxe, sigma=1, lam=1.0, mode="full", tier=0)
        assert r["n_maps"] == len(want) == g.count_maps(pxl, pxe)


def test_parallel_mining_driver_equals_serial_oracle():
    # the multi-process driver (all-cores CPU baseline, large parity samples) must return what
    # the oracle's own serial mining loop returns
    from oracle.parallel import Pool, mine_parallel
    cases = mining_cases(6, 77)
    pool = None
    try:
        for lab, src, dst, sigma, lam, max_edges, s in cases:
            if pool is not None:
                pool.close()
            pool = Pool(lab, src, dst, workers=2, seed=s)
            got = mine_parallel(pool, lab, src, dst, sigma, int(round(lam * 10**6)), max_edges)
            want = oracle.Graph(lab, src, dst, seed=s).mine(sigma=sigma, lam=lam, max_edges=max_edges)
            assert got == want
    finally:
        if pool is not None:
            pool.close()


# ----------------------------------------------------------------------------- directed graphs

def directed_cases(count, seed):
    st = Stream(seed)
    out = []
    for _ in range(count):
        nv = 5 + int(st.integers(1, 5)[0])
        na = nv + int(st.integers(1, 2 * nv)[0])
        s = int(st.next(1)[0] % (1 << 31))
        src = st.integers(na, nv).astype(np.int32)
        dst = st.integers(na, nv).astype(np.int32)
        lab = labels_uniform(nv, 1 + int(st.integers(1, 2)[0]), s + 1)
        n = 2 + int(st.integers(1, 3)[0])
        # a random weakly connected pattern: a random tree, each edge oriented at random, plus
        # a few extra arcs (reciprocal ones included)
        pe = pattern_edges("tree", n, st)
        arcs = [(a, b) if st.uniform(1)[0] < 0.5 else (b, a) for a, b in pe]
        for _ in range(int(st.integers(1, 3)[0])):
            a, b = (int(x) for x in st.integers(2, n))
            if a != b and (a, b) not in arcs:
                arcs.append((a, b))
        pl = [int(x) for x in st.integers(n, int(lab.max()) + 1)]
        out.append((lab, src, dst, pl, arcs, s))
    return out


def test_directed_tiers_agree_with_brute_force():
    for lab, src, dst, pl, arcs, s in directed_cases(100, 41):
        A = list(zip(src.tolist(), dst.tolist()))
        M = bf.maps_directed(lab.tolist(), A, pl, arcs)
        g = oracle.Graph(lab, src, dst, seed=s, directed=True)
        for sigma, lam in ((1, 1.0), (3, 0.5)):
            r0 = g.support(pl, arcs, sigma=sigma, lam=lam, mode="full", tier=0, want_selected=True)
            r1 = g.support(pl, arcs, sigma=sigma, lam=lam, mode="full", tier=1, want_selected=True)
            assert r0["n_maps"] == len(M) == g.count_maps(pl, arcs)
            assert (r0["mis"], r0["mni"], r0["selected"]) == (r1["mis"], r1["mni"], r1["selected"])
            assert r0["mni"] == bf.mni(M, len(pl))
            assert bf.is_independent(r1["selected"]) and bf.is_maximal(r1["selected"], M)


def test_directed_symmetric_graph_counts_equal_undirected():
    # both arcs of every edge + every pattern edge in both directions: the same maps as the
    # undirected graph and pattern (|M| and MNI agree; the greedy order need not)
    for lab, src, dst, pl, pe, s in tiny_cases(60, 43):
        both_s = np.concatenate([src, dst]).astype(np.int32)
        both_d = np.concatenate([dst, src]).astype(np.int32)
        arcs = [(a, b) for a, b in pe] + [(b, a) for a, b in pe]
        gd = oracle.Graph(lab, both_s, both_d, seed=s, directed=True)
        gu = oracle.Graph(lab, src, dst, seed=s)
        rd = gd.support(pl, arcs, sigma=1, lam=1.0, mode="full", tier=0)
        ru = gu.support(pl, pe, sigma=1, lam=1.0, mode="full", tier=0)
        assert (rd["n_maps"], rd["mni"]) == (ru["n_maps"], ru["mni"])


def test_directed_relabelling_invariance():
    st = Stream(45)
    for lab, src, dst, pl, arcs, s in directed_cases(40, 47):
        g = oracle.Graph(lab, src, dst, seed=s, directed=True)
        n = len(pl)
        perm = [int(x) for x in st.permutation(n)]
        pl2 = [0] * n
        for u in range(n):
            pl2[perm[u]] = pl[u]
        arcs2 = [(perm[a], perm[b]) for a, b in arcs]
        a = g.support(pl, arcs, sigma=2, lam=0.5, mode="full", tier=1, want_selected=True)
        b = g.support(pl2, arcs2, sigma=2, lam=0.5, mode="full", tier=1, want_selected=True)
        assert (a["mis"], a["mni"], a["selected"]) == (b["mis"], b["mni"], b["selected"])
