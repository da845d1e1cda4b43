"""The device-built graph layout (graph_build.cu) against the host-built one (graph.cpp).

The host builder's arrays are checked on the CPU (tests/host_graph_check.cpp); here the device
build of the same edge list must give the same four arrays bit for bit (records, label runs,
adjacency, the vertex index in greedy-root order), the same counts and the same error codes.
Cases: repeated and reversed edges, self-loops, isolated vertices, more than 64 labels (the
neighbour-label mask keeps ranks < 64 only), a single label, no edges, no vertices, the id root
order and another seed, and the MiCo- and YouTube-shaped graphs at full size.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import paper_2404_01585_gb300 as fx
from workloads import Stream, chung_lu, labels_zipf, make_graph

pytestmark = pytest.mark.gpu
PARTS = (fx.FLEXIS_LAYOUT_VREC, fx.FLEXIS_LAYOUT_RUNS, fx.FLEXIS_LAYOUT_ADJ, fx.FLEXIS_LAYOUT_LAB_VTX)
COUNTS = ("n_vertices", "n_arcs", "n_self_loops", "n_duplicates", "n_labels", "max_degree", "device_bytes")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def load(lab, src, dst, **kw):
    t0 = time.perf_counter()
    g = fx.Graph(lab, src, dst, **kw)
    return g, time.perf_counter() - t0


def assert_same_layout(lab, src, dst, **kw):
    gd, td = load(lab, src, dst, **kw)
    gh, th = load(lab, src, dst, host_build=1, **kw)
    di, hi = gd.info(), gh.info()
    assert di["built_on_device"] == 1 and hi["built_on_device"] == 0
    for k in COUNTS:
        assert di[k] == hi[k], k
    for part in PARTS:
        a, b = gd.layout(part), gh.layout(part)
        assert a.shape == b.shape and np.array_equal(a, b), part
    gd.close()
    gh.close()
    return di, td, th


def messy_graph(nv, ne, nl, seed):
    """Chung-Lu edges plus repeats (same and reversed direction), self-loops and isolated
    vertices (the top tenth of the ids gets no edge)."""
    st = Stream(seed)
    s0, d0 = chung_lu(int(nv * 0.9), ne, 2.3, seed)
    pick = st.integers(ne // 5, ne)
    rev = st.integers(ne // 5, ne)
    loops = st.integers(ne // 50, nv)
    src = np.concatenate([s0, s0[pick], d0[rev], loops]).astype(np.int32)
    dst = np.concatenate([d0, d0[pick], s0[rev], loops]).astype(np.int32)
    perm = st.permutation(src.size)
    return labels_zipf(nv, nl, 1.1, seed + 1), src[perm], dst[perm]


@pytest.mark.parametrize("nv,ne,nl,kw", [
    (3000, 20000, 12, {}),
    (3000, 20000, 12, {"root_order": 1}),
    (3000, 20000, 12, {"seed": 12345}),
    (5000, 30000, 100, {}),   # ranks >= 64 are left out of the neighbour-label mask
    (2000, 9000, 1, {}),
    (70000, 600000, 29, {}),  # several radix tiles per pass, three bytes of vertex id
])
def test_device_layout_equals_host_layout(nv, ne, nl, kw):
    lab, src, dst = messy_graph(nv, ne, nl, 4100 + nv + nl)
    info, _, _ = assert_same_layout(lab, src, dst, **kw)
    assert info["n_self_loops"] > 0 and info["n_duplicates"] > 0


def test_degenerate_graphs():
    lab = np.array([3, 1, 3, 3, 0], np.int32)
    assert_same_layout(lab, np.zeros(0, np.int32), np.zeros(0, np.int32))           # no edges
    assert_same_layout(lab, np.array([2, 2], np.int32), np.array([2, 2], np.int32))  # only self-loops
    assert_same_layout(lab, np.array([0, 1, 1, 0], np.int32), np.array([1, 0, 0, 1], np.int32))
    assert_same_layout(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))


def expect_error(code, lab, src, dst):
    for host in (0, 1):
        with pytest.raises(fx.FlexisError) as e:
            fx.Graph(lab, src, dst, host_build=host)
        assert e.value.code == code, host


def test_errors_match_host_build():
    lab = np.array([0, 1, 2, 1], np.int32)
    expect_error(fx.FLEXIS_E_INVALID, lab, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    expect_error(fx.FLEXIS_E_INVALID, lab, np.array([0, -1], np.int32), np.array([1, 2], np.int32))
    expect_error(fx.FLEXIS_E_INVALID, np.array([0, -2, 1], np.int32), np.array([0], np.int32), np.array([1], np.int32))
    many = np.arange(300, dtype=np.int32)  # 255 or more labels present: unsupported layout
    expect_error(fx.FLEXIS_E_UNSUPPORTED, many, np.array([0], np.int32), np.array([1], np.int32))
    # a bad endpoint is reported before the label count
    expect_error(fx.FLEXIS_E_INVALID, many, np.array([0], np.int32), np.array([300], np.int32))


@pytest.mark.parametrize("name", ["mico", "youtube"])
def test_full_size_layouts(name):
    lab, src, dst = make_graph(name)
    info, td, th = assert_same_layout(lab, src, dst)
    print(f"{name}: {info['n_vertices']} v, {info['n_arcs']} arcs: device build {td * 1e3:.1f} ms, "
          f"host build {th * 1e3:.1f} ms")


def test_degree_limit():
    # a star whose centre has 2^24 neighbours: beyond the run-entry offset field on both sides
    n = (1 << 24) + 1
    lab = np.zeros(n, np.int32)
    src = np.zeros(n - 1, np.int32)
    dst = np.arange(1, n, dtype=np.int32)
    expect_error(fx.FLEXIS_E_UNSUPPORTED, lab, src, dst)
