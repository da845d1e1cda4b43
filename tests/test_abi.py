"""CPU-side checks of the C-ABI library: it loads, exports every symbol include/flexis.h declares,
and its host logic (canonical code, candidate generation, tau) agrees with the oracle.  No call
here touches a GPU."""
from __future__ import annotations

import os
import re

import numpy as np
import pytest

import oracle
import paper_2404_01585_gb300 as fx
from workloads import Stream

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2404_01585_gb300 import _build
    _build.build()
    oracle.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "flexis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(flexis_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 20
    L = fx.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(fx.SYMBOLS)


def test_struct_layouts_match_header(tmp_path):
    # the C compiler's view of every public struct (size and field offsets) against the binding's
    import ctypes as C
    import subprocess
    structs = [fx.flexis_options, fx.flexis_pattern, fx.flexis_support_result, fx.flexis_plan,
               fx.flexis_graph_info, fx.flexis_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "flexis.h"', 'int main(void) {']
    for st in structs:
        nm = st.__name__
        lines.append(f'printf("{nm} %zu\\n", sizeof({nm}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{nm}.{f} %zu\\n", offsetof({nm}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for st in structs:
        nm = st.__name__
        assert int(got[nm]) == C.sizeof(st), nm
        for f, _ in st._fields_:
            assert int(got[f"{nm}.{f}"]) == getattr(st, f).offset, (nm, f)
    assert C.sizeof(fx.flexis_plan) == 1024


def test_status_strings():
    assert fx.status_string(0) == "ok"
    assert fx.status_string(fx.FLEXIS_E_INVALID) == "invalid argument"


def random_patterns(count, seed, max_n=7, labels=3):
    st = Stream(seed)
    out = []
    for _ in range(count):
        n = 2 + int(st.integers(1, max_n - 1)[0])
        e = [(i, j) for i in range(n) for j in range(i + 1, n) if st.uniform(1)[0] < 0.45]
        lab = [int(x) for x in st.integers(n, labels)]
        out.append((lab, e))
    return out


def test_canonical_code_matches_oracle():
    for lab, e in random_patterns(400, 3, max_n=8):
        a = fx.canonical_code(lab, e)
        b = oracle.canonical(lab, e)
        assert a[:2] == b[:2]


def test_canonical_code_of_symmetric_patterns_matches_oracle():
    # stars, cliques, cycles, complete bipartite graphs and their one-label / two-label versions
    # have many twins and automorphisms (the search skips twins)
    st = Stream(77)
    shapes = []
    for n in range(2, 9):
        shapes.append((n, [(0, i) for i in range(1, n)]))
        shapes.append((n, [(i, j) for i in range(n) for j in range(i + 1, n)]))
        if n >= 3:
            shapes.append((n, [(i, (i + 1) % n) for i in range(n)]))
        for k in range(1, n):
            shapes.append((n, [(i, j) for i in range(k) for j in range(k, n)]))
    for n, e in shapes:
        for labels in (1, 2, 3):
            for _ in range(4):
                lab = [int(x) for x in st.integers(n, labels)]
                perm = [int(x) for x in st.permutation(n)]
                pe = [(perm[a], perm[b]) for a, b in e]
                pl = [0] * n
                for u in range(n):
                    pl[perm[u]] = lab[u]
                a = fx.canonical_code(pl, pe)
                b = oracle.canonical(pl, pe)
                assert a[:2] == b[:2], (pl, pe)
                # the returned order realises the code
                order = list(a[2])
                assert sorted(order) == list(range(n))
                assert [pl[v] for v in order] == list(a[0])
                adj = {(x, y) for x, y in pe} | {(y, x) for x, y in pe}
                bits, t = 0, 0
                for j in range(1, n):
                    for i in range(j):
                        bits = (bits << 1) | (0 if (order[i], order[j]) in adj else 1)
                assert bits == a[1]


def test_candidate_generation_paper_figures():
    R, B, G, Y = 0, 1, 2, 3
    tri = [(0, 1), (1, 2), (0, 2)]
    for F in ([([R, B, R], tri), ([B, B, R], tri)],
              [([B, R, R, R], [(0, 1), (1, 2), (0, 2), (1, 3)])],
              [([R, G, B], tri), ([R, G, Y], tri), ([R, B, Y], tri), ([G, B, Y], tri)],
              [([R, G, B], tri), ([R, G, Y], tri), ([R, B, Y], tri)]):
        assert fx.generate_candidates(F) == oracle.candidates(F)


def _connected(n, e):
    adj = {i: set() for i in range(n)}
    for a, b in e:
        adj[a].add(b)
        adj[b].add(a)
    seen = {0}
    st = [0]
    while st:
        u = st.pop()
        for v in adj[u] - seen:
            seen.add(v)
            st.append(v)
    return len(seen) == n


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_candidate_generation_matches_oracle_predicate(k):
    # merge-based generator (Algorithms 2-4) == predicate form, on random frequent sets
    st = Stream(100 + k)
    for trial in range(4):
        F = []
        seen = set()
        for _attempt in range(400):
            if len(F) >= 14:
                break
            n = k - 1
            e = [(i, j) for i in range(n) for j in range(i + 1, n) if st.uniform(1)[0] < 0.5]
            if not e or not _connected(n, e):
                continue
            lab = [int(x) for x in st.integers(n, 2)]
            c = oracle.canonical(lab, e)[:2]
            if c in seen:
                continue
            seen.add(c)
            F.append((lab, e))
        for me in (0, k + 1):
            assert fx.generate_candidates(F, me) == oracle.candidates(F, me)


def test_lambda_quantisation_rounds_half_away_from_zero():
    # lambda -> num / 10^6 with num = llround(lambda * 10^6): the double product rounded to the
    # nearest integer, halves away from zero (the binding no longer rounds on its own)
    from decimal import ROUND_HALF_UP, Decimal
    st = Stream(31)
    vals = [0.0, 1.0, 0.5, 0.25, 2.5e-6, 0.0000125, 0.1234565, 0.9999995] + list(st.uniform(200))
    for lam in vals:
        want = int(Decimal(float(lam) * 1e6).quantize(Decimal(1), rounding=ROUND_HALF_UP))
        assert fx.lambda_quantize(float(lam)) == want, lam
    for bad in (-1e-9, 1.0000001, float("nan")):
        with pytest.raises(fx.FlexisError):
            fx.lambda_quantize(bad)
