"""GPU parity: the CUDA path (through the C ABI) against the oracle, element by element.

All quantities are integers, so the bar is bit-exact: mis, mni, tau, the frequent flag, the
selected maps themselves, and the frequent-pattern sets of mining."""
from __future__ import annotations

import json
import os
import time

import numpy as np
import pytest

import oracle
import paper_2404_01585_gb300 as fx
from tests.test_oracle import tiny_cases
from workloads import make_graph, random_patterns

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
EARLY, FULL = fx.FLEXIS_MODE_EARLY, fx.FLEXIS_MODE_FULL
SHAPES = ["tree", "cycle", "clique", "path", "star"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def key(r):
    return (r["tau"], r["mis"], r["mni"], bool(r["frequent"]))


def check_batch(g, og, pats, sigma, lam, mode, tier=1):
    res = g.support_batch(pats, sigma, lam, mode)
    m = "early" if mode == EARLY else "full"
    for (pl, pe), r in zip(pats, res):
        assert r["status"] == 0
        w = og.support(pl, pe, sigma=sigma, lam=lam, mode=m, tier=tier)
        assert key(r) == (w["tau"], w["mis"], w["mni"], w["frequent"]), (pl, pe, r, w)
    return res


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_running_example_all_seeds():
    d = load("running_example.json")
    e = np.asarray(d["data_edges"])
    for seed in range(32):
        g = fx.Graph(d["data_labels"], e[:, 0], e[:, 1], seed=seed, record_selected=16)
        og = oracle.Graph(d["data_labels"], e[:, 0], e[:, 1], seed=seed)
        for P in (d["P1"], d["P2"]):
            for mode, m in ((FULL, "full"), (EARLY, "early")):
                for sigma, lam in ((2, 1.0), (2, 0.25), (3, 1.0)):
                    r = g.support(P["labels"], P["edges"], sigma, lam, mode=mode)
                    w = og.support(P["labels"], P["edges"], sigma=sigma, lam=lam, mode=m, tier=0,
                                   want_selected=True)
                    assert key(r) == (w["tau"], w["mis"], w["mni"], w["frequent"])
                    assert g.selected_maps(0, 3) == w["selected"][: r["mis"]]
        g.close()


def test_theorem1_example_all_seeds():
    d = load("malvisual.json")
    e = np.asarray(d["data_edges"])
    for seed in range(64):
        g = fx.Graph(d["data_labels"], e[:, 0], e[:, 1], seed=seed, record_selected=16)
        og = oracle.Graph(d["data_labels"], e[:, 0], e[:, 1], seed=seed)
        r = g.support(d["P"]["labels"], d["P"]["edges"], 1, 1.0, mode=FULL)
        w = og.support(d["P"]["labels"], d["P"]["edges"], sigma=1, lam=1.0, mode="full", tier=0,
                       want_selected=True)
        assert (r["mis"], r["mni"]) == (w["mis"], w["mni"]) and r["mni"] == 5
        assert g.selected_maps(0, 4) == w["selected"]
        g.close()


def test_tiny_random_graphs_exhaustive_oracle():
    for lab, src, dst, pl, pe, s in tiny_cases(120, 17):
        g = fx.Graph(lab, src, dst, seed=s)
        og = oracle.Graph(lab, src, dst, seed=s)
        for mode in (FULL, EARLY):
            for sigma, lam in ((1, 1.0), (3, 0.5), (5, 0.0)):
                check_batch(g, og, [(pl, pe)], sigma, lam, mode, tier=0)
        g.close()


@pytest.fixture(scope="module")
def powerlaw():
    # sizes the plain oracle finishes in seconds: its depth-first search has no backjumping, and
    # 7-8 vertex trees and cycles through the hubs of this graph take it minutes
    lab, src, dst = make_graph(kind="cl", nv=20000, ne=100000, nl=8, law="zipf", zipf_s=1.0,
                               gamma=2.3, seed=41)
    pats = random_patterns(80, range(2, 7), SHAPES, lab, 43)
    return lab, src, dst, pats


@pytest.fixture(scope="module")
def er_large_patterns():
    # 7 and 8 vertex patterns on a graph without hubs (the oracle stays fast)
    lab, src, dst = make_graph(kind="er", nv=6000, ne=30000, nl=4, law="uniform", zipf_s=None,
                               gamma=None, seed=47)
    pats = random_patterns(40, range(7, 9), SHAPES, lab, 49)
    return lab, src, dst, pats


@pytest.mark.parametrize("mode", [EARLY, FULL])
def test_large_patterns_vs_oracle(er_large_patterns, mode):
    lab, src, dst, pats = er_large_patterns
    g = fx.Graph(lab, src, dst)
    og = oracle.Graph(lab, src, dst)
    for sigma, lam in ((30, 0.5), (2, 0.0)):
        check_batch(g, og, pats, sigma, lam, mode)
    g.close()


@pytest.mark.parametrize("mode", [EARLY, FULL])
@pytest.mark.parametrize("budget", [0, 2])
def test_powerlaw_batch_vs_oracle(powerlaw, mode, budget):
    lab, src, dst, pats = powerlaw
    g = fx.Graph(lab, src, dst, search_budget=budget)
    og = oracle.Graph(lab, src, dst)
    for sigma, lam in ((60, 0.5), (400, 1.0), (5, 0.0)):
        check_batch(g, og, pats, sigma, lam, mode)
    g.close()


def test_plain_equals_batched_and_launch_shape_free(powerlaw):
    lab, src, dst, pats = powerlaw
    ref = None
    for opts in ({}, dict(window_min=1, window_max=32), dict(window_min=1024, window_max=1024),
                 dict(search_blocks=3), dict(window_min=7, window_max=64, search_blocks=151),
                 dict(search_budget=1), dict(search_budget=3, window_min=4096, window_max=16384),
                 dict(search_budget=-1), dict(graphs=-1), dict(timing=1), dict(graphs=-1, timing=1)):
        g = fx.Graph(lab, src, dst, **opts)
        for mode in (EARLY, FULL):
            batch = [key(r) for r in g.support_batch(pats, 60, 0.5, mode)]
            # the round loop is replayed as a captured CUDA graph unless turned off
            assert (g.stats()["graph_launches"] > 0) == (opts.get("graphs", 0) >= 0), opts
            if ref is None:
                ref = {}
            if mode not in ref:
                ref[mode] = batch
            assert batch == ref[mode], opts
        plain = [key(g.support(pl, pe, 60, 0.5, mode=EARLY)) for pl, pe in pats[:12]]
        assert plain == ref[EARLY][:12]
        g.close()


@pytest.mark.parametrize("budget", [0, 1])
def test_selected_maps_equal_oracle(powerlaw, budget):
    # budget 1: every root search is suspended after each candidate chunk and resumed in the next
    # round under a grown used set
    lab, src, dst, pats = powerlaw
    g = fx.Graph(lab, src, dst, record_selected=4096, search_budget=budget)
    og = oracle.Graph(lab, src, dst)
    res = g.support_batch(pats[:30], 60, 0.5, FULL)
    for i, ((pl, pe), r) in enumerate(zip(pats[:30], res)):
        w = og.support(pl, pe, sigma=60, lam=0.5, mode="full", tier=1, want_selected=True)
        assert r["mis"] == w["mis"]
        assert g.selected_maps(i, len(pl), 4096) == w["selected"][:4096]
    g.close()


def test_edge_cases():
    lab, src, dst = make_graph(kind="er", nv=500, ne=1500, nl=3, law="uniform", zipf_s=None,
                               gamma=None, seed=5)
    g = fx.Graph(lab, src, dst)
    og = oracle.Graph(lab, src, dst)
    # label absent from the graph: no map at all
    r = g.support([0, 7], [(0, 1)], 1, 1.0, mode=FULL)
    assert (r["mis"], r["mni"], r["frequent"]) == (0, 0, False) and r["flags"] & fx.FLEXIS_FLAG_ABSENT_LABEL
    # invalid: disconnected pattern, n = 1, n = 9, lambda out of range, sigma < 1
    for bad in (([0, 1, 2], [(0, 1)]), ([0], []), ([0] * 9, [(i, i + 1) for i in range(8)])):
        with pytest.raises(fx.FlexisError):
            g.support(bad[0], bad[1], 5, 0.5)
    with pytest.raises(fx.FlexisError):
        g.support([0, 1], [(0, 1)], 5, 1.5)
    with pytest.raises(fx.FlexisError):
        g.support([0, 1], [(0, 1)], 0, 0.5)
    # per-pattern errors inside a batch do not fail the batch
    res = g.support_batch([([0, 1], [(0, 1)]), ([0, 1, 2], [(0, 1)])], 5, 0.5)
    assert res[0]["status"] == 0 and res[1]["status"] == fx.FLEXIS_E_INVALID
    # n = 2 and n = 8, sigma far above anything, tau = 0 (cap 1)
    pats = [([0, 1], [(0, 1)]), ([0] * 8, [(i, j) for i in range(8) for j in range(i + 1, 8)]),
            ([0, 1, 2, 0, 1, 2, 0, 1], [(i, i + 1) for i in range(7)])]
    for sigma, lam in ((1, 0.0), (2, 0.0), (10**9, 1.0), (7, 0.3)):
        for mode in (EARLY, FULL):
            check_batch(g, og, pats, sigma, lam, mode)
    g.close()
    # graph with isolated vertices and no edges
    g = fx.Graph([0, 1, 0, 1], [], [])
    r = g.support([0, 1], [(0, 1)], 1, 1.0, mode=FULL)
    assert (r["mis"], r["mni"]) == (0, 0)
    g.close()


def test_mine_citeseer_shape():
    lab, src, dst = make_graph("citeseer")
    g = fx.Graph(lab, src, dst)
    og = oracle.Graph(lab, src, dst)
    for sigma, lam, me in ((300, 0.5, 4), (30, 0.5, 4), (60, 0.0, 3)):
        got, glev = g.mine(sigma, lam, me)
        want, wlev = og.mine(sigma=sigma, lam=lam, max_edges=me)
        assert glev == wlev
        assert [(p["n"], p["code_labels"], p["code_bits"], p["tau"], p["mis"], p["mni"]) for p in got] == want
    g.close()


@pytest.mark.parametrize("budget", [0, 1])
def test_mine_small_powerlaw(powerlaw, budget):
    lab, src, dst, _ = powerlaw
    g = fx.Graph(lab, src, dst, search_budget=budget)
    og = oracle.Graph(lab, src, dst)
    got, glev = g.mine(300, 0.5, 3)
    want, wlev = og.mine(sigma=300, lam=0.5, max_edges=3)
    assert glev == wlev
    assert [(p["n"], p["code_labels"], p["code_bits"], p["tau"], p["mis"], p["mni"]) for p in got] == want
    g.close()


def test_serving_alone_equals_mixed(powerlaw):
    lab, src, dst, pats = powerlaw
    g = fx.Graph(lab, src, dst)
    alone = [key(r) for r in g.support_batch(pats, 60, 0.5, EARLY)]
    srv = fx.Server(g, slots=16)
    import time
    got = {}
    for i, (pl, pe) in enumerate(pats):
        assert srv.submit(i, pl, pe, 60, 0.5) == 0
        if i % 7 == 0:
            time.sleep(0.002)
        for rid, r, lat in srv.poll():
            got[rid] = r
    t0 = time.time()
    while len(got) < len(pats) and time.time() - t0 < 120:
        for rid, r, lat in srv.poll():
            got[rid] = r
        time.sleep(0.001)
    srv.stop()
    assert [key(got[i]) for i in range(len(pats))] == alone
    g.close()


def test_deadline_stops_undecided_patterns_only(powerlaw):
    # one-root windows make every pattern take a round per root, so a 1 ms limit passes while
    # many patterns are undecided; the decided ones keep their exact values
    lab, src, dst, pats = powerlaw
    # a pattern whose label is absent is decided before any round: one that always finishes
    pats = list(pats) + [([int(lab.max()) + 5, 0], [(0, 1)])]
    NO_MNI = fx.FLEXIS_MODE_NO_MNI
    g0 = fx.Graph(lab, src, dst)
    ref = g0.support_batch(pats, 60, 0.5, EARLY | NO_MNI)
    ref_full = g0.support_batch(pats, 60, 0.5, FULL)
    g0.close()
    g = fx.Graph(lab, src, dst, window_min=1, window_max=32, deadline_ms=1)
    res = g.support_batch(pats, 60, 0.5, EARLY | NO_MNI)
    stopped = 0
    for r, w in zip(res, ref):
        if r["status"] == fx.FLEXIS_E_TIMEOUT:
            stopped += 1
            assert 0 <= r["mis"] <= w["mis"] and r["mni"] == -1 and not r["frequent"]
        else:
            assert r["status"] == 0 and key(r) == key(w)
    assert 0 < stopped < len(pats)
    # the MNI pass checks the deadline too: a pattern stopped there keeps its final mis and
    # decision (only mni is missing); one stopped in its greedy phase is undecided
    for r, w in zip(g.support_batch(pats, 60, 0.5, FULL), ref_full):
        if r["status"] == fx.FLEXIS_E_TIMEOUT:
            assert r["mni"] == -1
            assert (r["mis"], r["frequent"]) == (w["mis"], w["frequent"]) or (r["mis"] <= w["mis"] and not r["frequent"])
        else:
            assert key(r) == key(w)
    with pytest.raises(fx.FlexisError) as e:
        g.mine(30, 0.5, 4)
    assert e.value.code == fx.FLEXIS_E_TIMEOUT
    # served requests: the limit runs from submission
    srv = fx.Server(g, slots=8)
    for i, (pl, pe) in enumerate(pats[:24]):
        assert srv.submit(i, pl, pe, 60, 0.5, EARLY | NO_MNI) == 0
    got, t0 = {}, time.time()
    while len(got) < 24 and time.time() - t0 < 120:
        for rid, r, lat in srv.poll():
            got[rid] = r
        time.sleep(0.001)
    srv.stop()
    assert len(got) == 24
    for i in range(24):
        r = got[i]
        assert r["status"] in (0, fx.FLEXIS_E_TIMEOUT)
        if r["status"] == 0:
            assert key(r) == key(ref[i])
    assert any(got[i]["status"] == fx.FLEXIS_E_TIMEOUT for i in range(24))
    g.close()


def test_used_bitmaps_left_clean_between_calls():
    # each evaluation clears only the used-bitmap words it dirtied (or its whole bitmap when it
    # dirtied more than it can list): results of later calls on the same workspace must equal
    # those of a fresh graph.  Exact full-mode counts of small patterns on 60k vertices dirty
    # every word of their bitmaps (the overflow path); the early-mode batch lists its words.
    lab, src, dst = make_graph(kind="cl", nv=60000, ne=300000, nl=4, law="zipf", zipf_s=1.0,
                               gamma=2.3, seed=53)
    big = random_patterns(24, range(2, 4), ["tree"], lab, 55)
    small = random_patterns(60, range(3, 6), SHAPES, lab, 57)
    full = FULL | fx.FLEXIS_MODE_NO_MNI
    g = fx.Graph(lab, src, dst)
    r1 = [key(r) for r in g.support_batch(big, 1, 0.0, full)]
    # >= 8192 used vertices over 1875 bitmap words: nearly every word is dirtied, more than the
    # 1024 a pattern's list holds
    assert max(r[1] for r in r1) > 4096
    r2 = [key(r) for r in g.support_batch(small, 40, 0.5, EARLY)]
    r3 = [key(r) for r in g.support_batch(big, 1, 0.0, full)]
    r4 = [key(r) for r in g.support_batch(small[:7], 40, 0.5, EARLY)]
    g.close()
    g2 = fx.Graph(lab, src, dst)
    assert r2 == [key(r) for r in g2.support_batch(small, 40, 0.5, EARLY)]
    assert r3 == r1 and r4 == r2[:7]
    g2.close()


def test_id_root_order_vs_oracle(powerlaw):
    # the root-order variant (roots by vertex id): tiny graphs against the brute-force tier, the
    # power-law batch against the backtracking tier, selected maps one by one
    for lab, src, dst, pl, pe, s in tiny_cases(40, 23):
        g = fx.Graph(lab, src, dst, seed=s, root_order=1)
        og = oracle.Graph(lab, src, dst, seed=s, root_order="id")
        for mode in (FULL, EARLY):
            check_batch(g, og, [(pl, pe)], 3, 0.5, mode, tier=0)
        g.close()
    lab, src, dst, pats = powerlaw
    g = fx.Graph(lab, src, dst, root_order=1, record_selected=4096)
    og = oracle.Graph(lab, src, dst, root_order="id")
    check_batch(g, og, pats, 60, 0.5, FULL)
    for i in range(0, 30, 3):
        pl, pe = pats[i]
        w = og.support(pl, pe, sigma=60, lam=0.5, mode="full", tier=1, want_selected=True)
        assert g.selected_maps(i, len(pl), 4096) == w["selected"][:4096]
    g.close()


def test_no_mni_mode(powerlaw):
    lab, src, dst, pats = powerlaw
    g = fx.Graph(lab, src, dst)
    og = oracle.Graph(lab, src, dst)
    res = g.support_batch(pats, 60, 0.5, EARLY | fx.FLEXIS_MODE_NO_MNI)
    for (pl, pe), r in zip(pats, res):
        w = og.support(pl, pe, sigma=60, lam=0.5, mode="early", tier=1)
        assert (r["tau"], r["mis"], bool(r["frequent"])) == (w["tau"], w["mis"], w["frequent"])
        assert r["mni"] == -1 and r["flags"] & fx.FLEXIS_FLAG_MNI_SKIPPED
    g.close()


def test_large_batch_active_list():
    # more patterns than the dense-commit threshold (4 blocks per SM): the commit kernel walks the
    # list of patterns still in their greedy phase
    lab, src, dst = make_graph(kind="cl", nv=4000, ne=16000, nl=5, law="zipf", zipf_s=1.0, gamma=2.3,
                               seed=61)
    pats = random_patterns(1500, range(2, 6), SHAPES, lab, 63)
    og = oracle.Graph(lab, src, dst)
    # window_max <= 1024 selects the small-horizon commit (at most 128 maps per pattern and
    # round); 1024-slot windows from the start make that horizon bind
    for opts in ({}, dict(search_budget=2, window_max=64), dict(window_min=1024, window_max=1024)):
        g = fx.Graph(lab, src, dst, **opts)
        check_batch(g, og, pats, 20, 0.5, EARLY)
        g.close()


def test_autotuner_results_identical_and_cached(powerlaw):
    # the measured autotuner times slices of a large batch under several search budgets; any
    # budget gives the same results, and the choice is kept for later batches of the same size
    lab, src, dst, _ = powerlaw
    pats = random_patterns(4500, range(2, 7), SHAPES, lab, 97)
    off = fx.Graph(lab, src, dst, autotune=-1)
    want = [key(r) for r in off.support_batch(pats, 60, 0.5, EARLY | fx.FLEXIS_MODE_NO_MNI)]
    assert off.stats()["autotune_probes"] == 0
    off.close()
    g = fx.Graph(lab, src, dst)
    first = [key(r) for r in g.support_batch(pats, 60, 0.5, EARLY | fx.FLEXIS_MODE_NO_MNI)]
    st = g.stats()
    assert st["autotune_probes"] == 3 and st["search_budget"] in (1024, 4096, 16384)
    second = [key(r) for r in g.support_batch(pats, 60, 0.5, EARLY | fx.FLEXIS_MODE_NO_MNI)]
    assert g.stats()["autotune_probes"] == 0 and g.stats()["search_budget"] == st["search_budget"]
    assert first == want and second == want
    g.close()
