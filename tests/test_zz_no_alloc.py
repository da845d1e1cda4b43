"""The allocation-free entry point (flexis_support_noalloc) gives the same supports as
flexis_support.

It serves callers that cannot call cudaMalloc while evaluating: its device scratch is one static
device array shared by every call on a GPU, so this file runs last (pytest collects it last) and
calls the entry point twice in a row to check that the second call starts from a clean state
although the array keeps the first call's contents."""
from __future__ import annotations

import pytest

import paper_2404_01585_gb300 as fx
from workloads import make_graph, random_patterns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def key(r):
    return (r["status"], r["tau"], r["mis"], r["mni"], bool(r["frequent"]))


def test_noalloc_matches_support_on_two_calls_in_a_row():
    lab, src, dst = make_graph(kind="cl", nv=20000, ne=100000, nl=8, law="zipf", zipf_s=1.0,
                               gamma=2.3, seed=41)
    g = fx.Graph(lab, src, dst)
    pats = random_patterns(12, range(3, 7), ["tree", "cycle", "clique", "path", "star"], lab, 91)
    for mode in (fx.FLEXIS_MODE_EARLY, fx.FLEXIS_MODE_FULL):
        plans = g.compile(pats, 60, 0.5, mode)
        for i, (pl, pe) in enumerate(pats):
            want = g.support(pl, pe, 60, 0.5, mode=mode)
            first = g.support_noalloc(plans[i])
            second = g.support_noalloc(plans[i])
            assert key(first) == key(want), (pl, pe, first, want)
            assert key(second) == key(want), (pl, pe, second, want)
    g.close()
