"""GPU parity on edge-labelled data graphs (Sec. 2.3.5, extended core graphs): the library's
extended graph and extended patterns (flexis_load_graph_edge_labels, flexis_pattern.edge_labels)
against the oracle run on the same extension written out independently in tests/bruteforce.py.
Bit-exact: tau, mis, mni, frequent, n_maps."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2404_01585_gb300 as fx
from tests import bruteforce as bf
from tests.test_oracle import edge_labelled_cases
from workloads import Stream, make_graph, random_patterns

pytestmark = pytest.mark.gpu
EARLY, FULL, COUNT = fx.FLEXIS_MODE_EARLY, fx.FLEXIS_MODE_FULL, fx.FLEXIS_MODE_COUNT_MAPS


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def oracle_of(lab, src, dst, el, seed=0x5EED):
    E = list(zip(np.asarray(src).tolist(), np.asarray(dst).tolist()))
    xl, xe, base = bf.extend_graph(np.asarray(lab).tolist(), E, list(el))
    og = oracle.Graph(np.asarray(xl, np.int32), np.asarray([a for a, b in xe], np.int32),
                      np.asarray([b for a, b in xe], np.int32), seed=seed)
    return og, base


def key(r):
    return (r["tau"], r["mis"], r["mni"], bool(r["frequent"]))


def test_tiny_edge_labelled_graphs_vs_oracle():
    for lab, src, dst, el, pl, pe, pel, s in edge_labelled_cases(80, 31):
        g = fx.Graph(lab, src, dst, edge_labels=el, seed=s)
        og, base = oracle_of(lab, src, dst, el, seed=s)
        info = g.info()
        assert info["edge_label_base"] == base and info["n_input_vertices"] == len(lab)
        xl, xe = bf.extend_pattern(pl, pe, pel, base)
        for mode, m in ((FULL, "full"), (EARLY, "early")):
            for sigma, lam in ((1, 1.0), (3, 0.5)):
                r = g.support(pl, pe, sigma, lam, mode=mode | COUNT, edge_labels=pel)
                w = og.support(xl, xe, sigma=sigma, lam=lam, mode=m, tier=0)
                assert r["status"] == 0 and key(r) == (w["tau"], w["mis"], w["mni"], w["frequent"]), (pl, pe, pel)
                assert r["n_maps"] == w["n_maps"] and r["n"] == len(xl)
        g.close()


def test_edge_labelled_powerlaw_batch_vs_oracle():
    lab, src, dst = make_graph(kind="cl", nv=5000, ne=20000, nl=4, law="zipf", zipf_s=1.0, gamma=2.3, seed=61)
    st = Stream(62)
    el = st.integers(src.size, 3).astype(np.int32)
    g = fx.Graph(lab, src, dst, edge_labels=el)
    og, base = oracle_of(lab, src, dst, el)
    pats = []
    for pl, pe in random_patterns(40, range(2, 5), ["path", "star", "tree"], lab, 63):
        pe = [tuple(x) for x in np.asarray(pe).tolist()]
        if len(pl) + len(pe) <= 8:
            pats.append((list(pl), pe, [int(x) for x in st.integers(len(pe), 3)]))
    res = g.support_batch(pats, 20, 0.5, EARLY | COUNT)
    for (pl, pe, pel), r in zip(pats, res):
        xl, xe = bf.extend_pattern(pl, pe, pel, base)
        w = og.support(xl, xe, sigma=20, lam=0.5, mode="early", tier=1)
        assert key(r) == (w["tau"], w["mis"], w["mni"], w["frequent"]), (pl, pe, pel, r, w)
        assert r["n_maps"] == min(og.count_maps(xl, xe), 1 << 32)
    g.close()


def test_edge_label_pattern_errors():
    lab, src, dst = make_graph(kind="er", nv=200, ne=600, nl=2, law="uniform", zipf_s=None, gamma=None, seed=65)
    el = np.zeros(src.size, np.int32)
    g = fx.Graph(lab, src, dst, edge_labels=el)
    # missing edge labels, too large once extended, repeated edge
    assert g.support_batch([([0, 1], [(0, 1)])], 2, 0.5)[0]["status"] == fx.FLEXIS_E_INVALID
    big = ([0] * 5, [(0, 1), (1, 2), (2, 3), (3, 4)], [0] * 4)
    assert g.support_batch([big], 2, 0.5)[0]["status"] == fx.FLEXIS_E_INVALID
    rep = ([0, 1], [(0, 1), (1, 0)], [0, 0])
    assert g.support_batch([rep], 2, 0.5)[0]["status"] == fx.FLEXIS_E_INVALID
    g.close()
    plain = fx.Graph(lab, src, dst)
    assert plain.support_batch([([0, 1], [(0, 1)], [0])], 2, 0.5)[0]["status"] == fx.FLEXIS_E_INVALID
    assert plain.info()["edge_label_base"] == -1
    plain.close()
