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


@pytest.fixture(scope="module")
def graph_and_patterns():
    lab, src, dst = make_graph(kind="cl", nv=20000, ne=100000, nl=8, law="zipf", zipf_s=1.0,
                               gamma=2.3, seed=41)
    pats = random_patterns(12, range(3, 7), ["tree", "cycle", "clique", "path", "star"], lab, 91)
    return lab, src, dst, pats


def key(r):
    return (r["status"], r["tau"], r["mis"], r["mni"], bool(r["frequent"]))


def test_noalloc_matches_support_on_two_calls_in_a_row(graph_and_patterns):
    lab, src, dst, pats = graph_and_patterns
    g = fx.Graph(lab, src, dst)
    for mode in (fx.FLEXIS_MODE_EARLY, fx.FLEXIS_MODE_FULL):
        plans = g.compile(pats, 60, 0.5, mode)
        for i, (pl, pe) in enumerate(pats):
            want = g.support(pl, pe, 60, 0.5, mode=mode)
            first = g.support_noalloc(plans[i])
            second = g.support_noalloc(plans[i])
            assert key(first) == key(want), (pl, pe, first, want)
            assert key(second) == key(want), (pl, pe, second, want)
    g.close()


def test_noalloc_on_a_caller_stream(graph_and_patterns):
    # the caller passes its own stream (here one made by PyTorch); the call runs and synchronises
    # on it, and the results equal flexis_support's
    torch = pytest.importorskip("torch")
    lab, src, dst, pats = graph_and_patterns
    g = fx.Graph(lab, src, dst)
    s = torch.cuda.Stream()
    plans = g.compile(pats, 60, 0.5, fx.FLEXIS_MODE_FULL)
    for i, (pl, pe) in enumerate(pats):
        want = g.support(pl, pe, 60, 0.5, mode=fx.FLEXIS_MODE_FULL)
        for _ in range(2):
            got = g.support_noalloc(plans[i], stream=s.cuda_stream)
            assert key(got) == key(want), (pl, pe, got, want)
    g.close()


def test_noalloc_honours_the_deadline(graph_and_patterns):
    # with a 1 ms deadline a pattern either finishes with the unbounded values or stops undecided
    # (FLEXIS_E_TIMEOUT) with a lower bound of its mIS, exactly as flexis_support does
    lab, src, dst, pats = graph_and_patterns
    free = fx.Graph(lab, src, dst)
    want = [free.support(pl, pe, 60, 0.5, mode=fx.FLEXIS_MODE_EARLY) for pl, pe in pats]
    free.close()
    g = fx.Graph(lab, src, dst, deadline_ms=1)
    plans = g.compile(pats, 60, 0.5, fx.FLEXIS_MODE_EARLY)
    for i in range(len(pats)):
        got = g.support_noalloc(plans[i])
        if got["status"] == fx.FLEXIS_E_TIMEOUT:
            assert 0 <= got["mis"] <= want[i]["mis"] and not got["frequent"]
        else:
            assert key(got) == key(want[i])
    g.close()
