"""GPU parity on directed data graphs (the paper's matcher is directed, Sec. 2.2 / Sec. 4.1):
options.directed = 1, pattern edges read as arcs.  Bit-exact against the oracle's directed
graphs: tau, mis, mni, frequent, the selected maps, and n_maps."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2404_01585_gb300 as fx
from tests.test_oracle import directed_cases
from workloads import Stream, make_graph, pattern_edges

pytestmark = pytest.mark.gpu
EARLY, FULL, COUNT = fx.FLEXIS_MODE_EARLY, fx.FLEXIS_MODE_FULL, fx.FLEXIS_MODE_COUNT_MAPS


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def key(r):
    return (r["tau"], r["mis"], r["mni"], bool(r["frequent"]))


def test_tiny_directed_graphs_vs_oracle():
    for lab, src, dst, pl, arcs, s in directed_cases(100, 41):
        g = fx.Graph(lab, src, dst, seed=s, directed=1, record_selected=64)
        og = oracle.Graph(lab, src, dst, seed=s, directed=True)
        assert g.info()["directed"] == 1
        for mode, m in ((FULL, "full"), (EARLY, "early")):
            for sigma, lam in ((1, 1.0), (3, 0.5)):
                r = g.support(pl, arcs, sigma, lam, mode=mode | COUNT)
                w = og.support(pl, arcs, sigma=sigma, lam=lam, mode=m, tier=0, want_selected=True)
                assert r["status"] == 0 and key(r) == (w["tau"], w["mis"], w["mni"], w["frequent"]), (pl, arcs, r, w)
                assert r["n_maps"] == w["n_maps"]
                assert g.selected_maps(0, len(pl)) == w["selected"][: r["mis"]]
        g.close()


def directed_powerlaw(seed):
    lab, src, dst = make_graph(kind="cl", nv=20000, ne=100000, nl=6, law="zipf", zipf_s=1.0, gamma=2.3, seed=seed)
    st = Stream(seed + 1)
    flip = st.uniform(src.size) < 0.5
    s2 = np.where(flip, dst, src).astype(np.int32)
    d2 = np.where(flip, src, dst).astype(np.int32)
    # a fifth of the edges also get the reverse arc (mutual neighbours)
    back = st.uniform(src.size) < 0.2
    return lab, np.concatenate([s2, d2[back]]), np.concatenate([d2, s2[back]])


def random_directed_patterns(count, sizes, lab, seed):
    st = Stream(seed)
    out = []
    for _ in range(count):
        n = sizes[int(st.integers(1, len(sizes))[0])]
        shape = ("tree", "cycle", "path", "star")[int(st.integers(1, 4)[0])]
        pe = pattern_edges(shape, n, st)
        arcs = [(a, b) if st.uniform(1)[0] < 0.5 else (b, a) for a, b in pe]
        if st.uniform(1)[0] < 0.3:
            a, b = arcs[0]
            arcs.append((b, a))
        out.append((lab[st.integers(n, lab.size)].astype(np.int32).tolist(), arcs))
    return out


def test_directed_powerlaw_batch_vs_oracle():
    lab, src, dst = directed_powerlaw(71)
    pats = random_directed_patterns(60, [2, 3, 4, 5, 6], lab, 73)
    og = oracle.Graph(lab, src, dst, directed=True)
    for opts in ({}, dict(window_min=1, window_max=32, search_budget=2)):
        g = fx.Graph(lab, src, dst, directed=1, **opts)
        for mode, m in ((EARLY, "early"), (FULL, "full")):
            res = g.support_batch(pats, 40, 0.5, mode)
            for (pl, arcs), r in zip(pats, res):
                w = og.support(pl, arcs, sigma=40, lam=0.5, mode=m, tier=1)
                assert key(r) == (w["tau"], w["mis"], w["mni"], w["frequent"]), (pl, arcs, r, w, opts)
        g.close()


def test_directed_counts_and_mining_unsupported():
    lab, src, dst = directed_powerlaw(75)
    pats = random_directed_patterns(30, [3, 4, 5], lab, 77)
    og = oracle.Graph(lab, src, dst, directed=True)
    g = fx.Graph(lab, src, dst, directed=1, maps_cap=100000)
    res = g.support_batch(pats, 40, 0.5, EARLY | COUNT | fx.FLEXIS_MODE_NO_MNI)
    for (pl, arcs), r in zip(pats, res):
        assert r["n_maps"] == min(og.count_maps(pl, arcs, cap=100000), 100000), (pl, arcs, r)
    with pytest.raises(fx.FlexisError) as e:
        g.mine(40, 0.5, 3)
    assert e.value.code == fx.FLEXIS_E_UNSUPPORTED
    g.close()
