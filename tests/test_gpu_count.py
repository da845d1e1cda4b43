"""GPU parity of the map count (FLEXIS_MODE_COUNT_MAPS, the level-by-level enumerator) and of
the count-only mode (FLEXIS_MODE_COUNT_MAPS | FLEXIS_MODE_NO_MIS): n_maps = |M| (Sec. 2.4)
against the oracle's brute-force map list (tier 0) and its backtracking count, element by
element; integer work, so the bar is exact equality."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
import paper_2404_01585_gb300 as fx
from tests.test_oracle import tiny_cases
from workloads import make_graph, random_patterns

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
EARLY, FULL = fx.FLEXIS_MODE_EARLY, fx.FLEXIS_MODE_FULL
COUNT, NO_MIS = fx.FLEXIS_MODE_COUNT_MAPS, fx.FLEXIS_MODE_NO_MIS
SHAPES = ["tree", "cycle", "clique", "path", "star"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_running_example_six_maps():
    # Sec. 2.2 lists the six maps of P1 in D; P2 has four (derived by hand from Fig. 1)
    with open(os.path.join(GOLD, "running_example.json")) as f:
        d = json.load(f)
    e = np.asarray(d["data_edges"])
    g = fx.Graph(d["data_labels"], e[:, 0], e[:, 1])
    for P, want in ((d["P1"], len(d["P1_maps_u1u2u3"])), (d["P2"], d["P2_maps"])):
        for mode in (FULL | COUNT, EARLY | COUNT, FULL | COUNT | NO_MIS):
            r = g.support(P["labels"], P["edges"], 2, 1.0, mode=mode)
            assert r["status"] == 0 and r["n_maps"] == want, (P, mode, r)
            assert not r["flags"] & fx.FLEXIS_FLAG_MAPS_SATURATED
    r = g.support(d["P1"]["labels"], d["P1"]["edges"], 2, 1.0, mode=FULL | COUNT | NO_MIS)
    assert r["mis"] == -1 and r["mni"] == d["P1_MNI"] and r["flags"] & fx.FLEXIS_FLAG_MIS_SKIPPED
    # without the flag nothing is counted
    assert g.support(d["P1"]["labels"], d["P1"]["edges"], 2, 1.0, mode=FULL)["n_maps"] == 0
    g.close()


def test_tiny_graphs_count_equals_brute_force():
    for lab, src, dst, pl, pe, s in tiny_cases(120, 17):
        g = fx.Graph(lab, src, dst, seed=s)
        og = oracle.Graph(lab, src, dst, seed=s)
        w = og.support(pl, pe, sigma=3, lam=0.5, mode="full", tier=0)
        for mode in (FULL | COUNT, EARLY | COUNT):
            r = g.support_batch([(pl, pe)], 3, 0.5, mode)[0]
            assert r["n_maps"] == w["n_maps"], (pl, pe, r, w)
            m = "full" if mode & 3 == FULL else "early"
            w2 = og.support(pl, pe, sigma=3, lam=0.5, mode=m, tier=0)
            assert (r["tau"], r["mis"], r["mni"], bool(r["frequent"])) == (w2["tau"], w2["mis"], w2["mni"], w2["frequent"])
        c = g.support_batch([(pl, pe)], 3, 0.5, FULL | COUNT | NO_MIS)[0]
        assert (c["n_maps"], c["mis"], c["mni"], c["frequent"]) == (w["n_maps"], -1, w["mni"], False)
        g.close()


@pytest.fixture(scope="module")
def powerlaw():
    lab, src, dst = make_graph(kind="cl", nv=20000, ne=100000, nl=8, law="zipf", zipf_s=1.0,
                               gamma=2.3, seed=41)
    pats = random_patterns(40, range(2, 7), SHAPES, lab, 143)
    return lab, src, dst, pats


CAP = 200_000


def test_powerlaw_counts_vs_oracle_backtracking(powerlaw):
    # counts at or above the cap saturate on both sides (the oracle stops at the cap)
    lab, src, dst, pats = powerlaw
    og = oracle.Graph(lab, src, dst)
    want = [og.count_maps(pl, pe, cap=CAP) for pl, pe in pats]
    assert any(0 < x < CAP for x in want) and any(x >= CAP for x in want)
    for opts in ({}, dict(frontier_rows=64), dict(frontier_rows=1 << 16)):
        g = fx.Graph(lab, src, dst, maps_cap=CAP, **opts)
        res = g.support_batch(pats, 60, 0.5, EARLY | COUNT | fx.FLEXIS_MODE_NO_MNI)
        for (pl, pe), r, w in zip(pats, res, want):
            assert r["status"] == 0
            assert r["n_maps"] == min(w, CAP), (pl, pe, r, w, opts)
            assert bool(r["flags"] & fx.FLEXIS_FLAG_MAPS_SATURATED) == (w >= CAP), (pl, pe, r, w)
        g.close()


def test_count_only_mode_mni_exact(powerlaw):
    lab, src, dst, pats = powerlaw
    og = oracle.Graph(lab, src, dst)
    g = fx.Graph(lab, src, dst, maps_cap=CAP)
    small = pats[:16]
    res = g.support_batch(small, 60, 0.5, FULL | COUNT | NO_MIS)
    for (pl, pe), r in zip(small, res):
        w = og.support(pl, pe, sigma=60, lam=0.5, mode="full", tier=1)
        assert r["mis"] == -1 and r["mni"] == w["mni"] and not r["frequent"], (pl, pe, r, w)
        assert r["n_maps"] == min(og.count_maps(pl, pe, cap=CAP), CAP)
    g.close()


def test_er_large_patterns_counts():
    lab, src, dst = make_graph(kind="er", nv=6000, ne=30000, nl=4, law="uniform", zipf_s=None,
                               gamma=None, seed=47)
    pats = random_patterns(24, range(7, 9), SHAPES, lab, 149)
    og = oracle.Graph(lab, src, dst)
    g = fx.Graph(lab, src, dst, maps_cap=CAP)
    res = g.support_batch(pats, 30, 0.5, EARLY | COUNT)
    for (pl, pe), r in zip(pats, res):
        w = og.count_maps(pl, pe, cap=CAP)
        assert r["n_maps"] == min(w, CAP), (pl, pe, r, w)
    g.close()


def test_count_is_independent_of_the_batch(powerlaw):
    lab, src, dst, pats = powerlaw
    g = fx.Graph(lab, src, dst, maps_cap=CAP)
    batch = [r["n_maps"] for r in g.support_batch(pats, 60, 0.5, EARLY | COUNT)]
    single = [g.support(pl, pe, 60, 0.5, mode=EARLY | COUNT)["n_maps"] for pl, pe in pats[:10]]
    assert single == batch[:10]
    g.close()


# ----------------------------------------------------------------------------- overlap graph, MIS
EXACT = fx.FLEXIS_MODE_EXACT_MIS


def test_overlap_graph_and_exact_mis_paper_examples():
    with open(os.path.join(GOLD, "running_example.json")) as f:
        d = json.load(f)
    e = np.asarray(d["data_edges"])
    g = fx.Graph(d["data_labels"], e[:, 0], e[:, 1])
    inst, edges = g.overlap_graph(d["P1"]["labels"], d["P1"]["edges"])
    assert inst == [(0, 1, 4), (1, 2, 5), (2, 3, 6)] and edges == [(0, 1), (1, 2)]
    for mode in (FULL | EXACT, EARLY | EXACT, FULL | EXACT | NO_MIS | COUNT):
        r = g.support(d["P1"]["labels"], d["P1"]["edges"], 2, 1.0, mode=mode)
        assert r["mis_exact"] == d["P1_MIS"] == 2, (mode, r)
        assert not r["flags"] & fx.FLEXIS_FLAG_EXACT_MIS_SATURATED
    assert g.support(d["P1"]["labels"], d["P1"]["edges"], 2, 1.0, mode=FULL)["mis_exact"] == -1
    g.close()
    with open(os.path.join(GOLD, "malvisual.json")) as f:
        m = json.load(f)
    e = np.asarray(m["data_edges"])
    g = fx.Graph(m["data_labels"], e[:, 0], e[:, 1])
    r = g.support(m["P"]["labels"], m["P"]["edges"], 1, 1.0, mode=FULL | EXACT)
    assert r["mis_exact"] == m["MIS"] == 4 and r["mis"] <= 4 <= 4 * r["mis"]
    g.close()


def test_overlap_graph_and_exact_mis_tiny_graphs():
    seen = 0
    for lab, src, dst, pl, pe, s in tiny_cases(120, 23):
        g = fx.Graph(lab, src, dst, seed=s)
        og = oracle.Graph(lab, src, dst, seed=s)
        assert g.overlap_graph(pl, pe) == og.overlap_graph(pl, pe), (pl, pe)
        big = og.max_independent_set(pl, pe, max_inst=40)
        if big is not None:
            r = g.support_batch([(pl, pe)], 1, 1.0, FULL | EXACT)[0]
            assert r["mis_exact"] == big and not r["flags"] & fx.FLEXIS_FLAG_EXACT_MIS_SATURATED, (pl, pe, r, big)
            assert r["mis"] <= big <= len(pl) * r["mis"] or big == 0
            seen += 1
        g.close()
    assert seen >= 100


def test_exact_mis_sparse_graph_small_overlap_graphs():
    # overlap graphs small enough for the oracle's exhaustive search: a sparse graph, many labels
    lab, src, dst = make_graph(kind="er", nv=3000, ne=5000, nl=6, law="uniform", zipf_s=None,
                               gamma=None, seed=153)
    pats = random_patterns(300, range(2, 6), ["path", "star", "cycle", "tree"], lab, 151)
    og = oracle.Graph(lab, src, dst)
    small = []
    for pl, pe in pats:
        if og.count_maps(pl, pe, cap=5000) >= 5000:
            continue
        got = og.overlap_graph(pl, pe, max_maps=5000, cap_inst=30)
        if got is not None and 2 <= len(got[0]) <= 30:
            small.append((pl, pe, og.max_independent_set(pl, pe, max_maps=5000, max_inst=30), got))
    assert len(small) >= 10
    g = fx.Graph(lab, src, dst)
    res = g.support_batch([(pl, pe) for pl, pe, _, _ in small], 60, 0.5, FULL | EXACT | fx.FLEXIS_MODE_NO_MNI)
    for (pl, pe, big, got), r in zip(small, res):
        assert r["mis_exact"] == big, (pl, pe, r, big)
        assert g.overlap_graph(pl, pe) == got
    g.close()


def test_exact_mis_limits_give_a_flagged_lower_bound(powerlaw):
    lab, src, dst, pats = powerlaw
    g = fx.Graph(lab, src, dst, exact_mis_maps=8, exact_mis_nodes=50)
    res = g.support_batch(pats[:20], 60, 0.5, FULL | EXACT | fx.FLEXIS_MODE_NO_MNI)
    flagged = 0
    for r in res:
        assert r["status"] == 0 and r["mis_exact"] >= 0
        if r["flags"] & fx.FLEXIS_FLAG_EXACT_MIS_SATURATED:
            flagged += 1
            assert r["mis_exact"] >= r["mis"]  # never below the greedy's independent set
    assert flagged > 0
    g.close()
