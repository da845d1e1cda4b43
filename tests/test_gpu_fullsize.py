"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py times.

* MiCo-shaped graph (100,000 vertices, 1,080,000 edges, 29 labels), sigma = 3000 at lambda = 0.5
  and lambda = 0: the whole frequent-pattern set of the mining loop up to 3 edges equals the
  oracle's (exact, every pattern and value); up to 5 edges, a deterministic sample of the
  frequent patterns is re-evaluated by the oracle.
* The 1 M-vertex batched level (2,000 trees / cycles / cliques of 3-7 vertices): the oracle
  re-evaluates the patterns it finishes in seconds (<= 4 vertices); for every pattern the
  selected maps themselves are checked against properties that hold at any size -- each is a
  map (injective, label- and edge-preserving), the maps are vertex-disjoint, their number is the
  reported mis (capped at c), and the decision is mis >= c.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2404_01585_gb300 as fx
from workloads import batch_level_patterns, make_graph

pytestmark = pytest.mark.gpu
EARLY, NO_MNI = fx.FLEXIS_MODE_EARLY, fx.FLEXIS_MODE_NO_MNI


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def mico():
    return make_graph("mico")


@pytest.mark.parametrize("lam", [0.5, 0.0])
def test_mico_mining_exact_to_3_edges(mico, lam):
    lab, src, dst = mico
    g = fx.Graph(lab, src, dst)
    og = oracle.Graph(lab, src, dst)
    got, glev = g.mine(3000, lam, 3)
    want, wlev = og.mine(sigma=3000, lam=lam, max_edges=3)
    assert glev == wlev
    assert [(p["n"], p["code_labels"], p["code_bits"], p["tau"], p["mis"], p["mni"]) for p in got] == want
    g.close()


@pytest.mark.parametrize("lam", [0.5, 0.0])
def test_mico_mining_sampled_to_5_edges(mico, lam):
    lab, src, dst = mico
    g = fx.Graph(lab, src, dst)
    og = oracle.Graph(lab, src, dst)
    got, levels = g.mine(3000, lam, 5)
    assert levels[6][1] > 0  # the sweep really reaches 6-vertex patterns
    for p in got:
        assert p["mis"] == p["tau"] and p["mni"] == p["tau"]  # frequent: counts capped at tau
    sample = [p for p in got if p["n"] >= 5][::max(1, len([p for p in got if p["n"] >= 5]) // 12)][:12]
    for p in sample:
        w = og.support(list(p["labels"]), p["edges"], sigma=3000, lam=lam, mode="early", tier=1)
        assert (w["tau"], w["mis"], w["mni"], w["frequent"]) == (p["tau"], p["mis"], p["mni"], True), p
    g.close()


@pytest.fixture(scope="module")
def cl1m():
    lab, src, dst = make_graph("cl1m")
    return lab, src, dst, batch_level_patterns(lab, 2000)


def csr(nv, src, dst):
    a = np.concatenate([src, dst]).astype(np.int64)
    b = np.concatenate([dst, src]).astype(np.int64)
    key = np.unique(a * nv + b)
    return key


def test_cl1m_batch_sampled_and_selected_maps_valid(cl1m):
    lab, src, dst, pats = cl1m
    g = fx.Graph(lab, src, dst, record_selected=1024)
    res = g.support_batch(pats, 1000, 0.5, EARLY | NO_MNI)
    nv = lab.size
    keys = csr(nv, src, dst)
    # label ranks (ascending frequency, ties by id): the canonical form the maps are indexed by
    cnt = np.bincount(lab)
    order = sorted((l for l in range(cnt.size) if cnt[l] > 0), key=lambda l: (cnt[l], l))
    rank_of = np.full(cnt.size, -1, dtype=np.int64)
    rank_of[np.asarray(order)] = np.arange(len(order))
    lab_rank = rank_of[lab]
    n_checked = 0
    for i, ((pl, pe), r) in enumerate(zip(pats, res)):
        assert r["status"] == 0
        cap = max(r["tau"], 1)
        assert r["frequent"] == (r["mis"] >= cap) and r["mis"] <= cap
        if i % 4:  # the selected-map check on every fourth pattern keeps the test short
            continue
        n = len(pl)
        maps = np.asarray(g.selected_maps(i, n, 1024), dtype=np.int64).reshape(-1, n)
        assert maps.shape[0] == min(r["mis"], 1024)
        if maps.size == 0:
            continue
        # maps are indexed by the vertices of the pattern's canonical form over label ranks
        plan_labels, plan_bits, _ = fx.canonical_code([int(rank_of[int(x)]) for x in pl], pe)
        # injective and vertex-disjoint across maps
        flat = maps.reshape(-1)
        assert np.unique(flat).size == flat.size
        # label preserving, position by position
        assert np.all(lab_rank[maps] == np.asarray(plan_labels)[None, :])
        # edges of the canonical pattern (decoded from its code bits) land on data edges
        cedges, t = [], n * (n - 1) // 2 - 1
        for b in range(1, n):
            for a in range(b):
                if not (plan_bits >> t) & 1:
                    cedges.append((a, b))
                t -= 1
        for a, b in cedges:
            k = maps[:, a] * nv + maps[:, b]
            pos = np.searchsorted(keys, k)
            assert np.all(pos < keys.size) and np.all(keys[np.minimum(pos, keys.size - 1)] == k)
        n_checked += 1
    assert n_checked > 400
    # the oracle re-evaluates the small patterns it finishes in seconds
    og = oracle.Graph(lab, src, dst)
    small = [i for i, (pl, pe) in enumerate(pats) if len(pl) <= 4][:16]
    for i in small:
        pl, pe = pats[i]
        w = og.support(pl, pe, sigma=1000, lam=0.5, mode="early", tier=1)
        assert (w["tau"], w["mis"], w["frequent"]) == (res[i]["tau"], res[i]["mis"], res[i]["frequent"]), (pl, pe)
    g.close()
