"""Python wrapper of the plain C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline leg
are the only callers.  The product path never imports this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LAMBDA_DEN = 1_000_000


def build(force: bool = False) -> str:
    """Compile oracle.c with the host C compiler (plain -O2, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
            L.or_tau.restype = C.c_int64
            L.or_tau.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int32]
            L.or_hash.restype = C.c_uint64
            L.or_hash.argtypes = [C.c_uint64, C.c_int64]
            L.or_graph_new.restype = C.c_void_p
            L.or_graph_new.argtypes = [C.c_int64, i32p, C.c_int64, i32p, i32p, C.c_uint64]
            L.or_graph_new2.restype = C.c_void_p
            L.or_graph_new2.argtypes = [C.c_int64, i32p, C.c_int64, i32p, i32p, C.c_uint64, C.c_int]
            L.or_graph_free.argtypes = [C.c_void_p]
            L.or_graph_set_root_order.argtypes = [C.c_void_p, C.c_int]
            L.or_graph_arcs.restype = C.c_int64
            L.or_graph_arcs.argtypes = [C.c_void_p]
            L.or_graph_rank.restype = C.c_int32
            L.or_graph_rank.argtypes = [C.c_void_p, C.c_int32]
            L.or_canonical.restype = C.c_int
            L.or_canonical.argtypes = [C.c_int, i32p, C.c_int, i32p, i32p,
                                       C.POINTER(C.c_uint32), i32p]
            L.or_support.restype = C.c_int
            L.or_support.argtypes = [C.c_void_p, C.c_int, i32p, C.c_int, i32p, C.c_int64,
                                     C.c_int64, C.c_int64, C.c_int, C.c_int, i64p, C.c_void_p,
                                     C.c_int64, C.POINTER(C.c_int64)]
            L.or_support_budget.restype = C.c_int
            L.or_support_budget.argtypes = [C.c_void_p, C.c_int, i32p, C.c_int, i32p, C.c_int64,
                                            C.c_int64, C.c_int64, C.c_int, C.c_int, i64p, C.c_void_p,
                                            C.c_int64, C.POINTER(C.c_int64), C.c_int64]
            L.or_count_maps.restype = C.c_int64
            L.or_count_maps.argtypes = [C.c_void_p, C.c_int, i32p, C.c_int, i32p, C.c_int64]
            L.or_overlap_graph.restype = C.c_int
            L.or_overlap_graph.argtypes = [C.c_void_p, C.c_int, i32p, C.c_int, i32p, C.c_int64, i32p,
                                           C.c_int64, C.POINTER(C.c_int64), i32p, C.c_int64,
                                           C.POINTER(C.c_int64)]
            L.or_max_independent_set.restype = C.c_int64
            L.or_max_independent_set.argtypes = [C.c_void_p, C.c_int, i32p, C.c_int, i32p, C.c_int64,
                                                 C.c_int64]
            L.or_candidates.restype = C.c_int64
            L.or_candidates.argtypes = [C.c_int, i32p, i32p, i32p, i32p, C.c_int, i32p, i32p,
                                        u32p, C.c_int64]
            L.or_mine.restype = C.c_void_p
            L.or_mine.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int]
            L.or_mined_count.restype = C.c_int64
            L.or_mined_count.argtypes = [C.c_void_p]
            L.or_mined_get.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), i32p,
                                       C.POINTER(C.c_uint32), i64p]
            L.or_mined_levels.argtypes = [C.c_void_p, i64p, i64p]
            L.or_mined_free.argtypes = [C.c_void_p]
            _lib = L
    return _lib


def lam_q(lam: float) -> int:
    """lambda as the exact rational p / 10^6 with p = round(lambda * 10^6)."""
    return int(round(lam * LAMBDA_DEN))


def tau(sigma: int, lam: float, n: int) -> int:
    return int(lib().or_tau(sigma, lam_q(lam), LAMBDA_DEN, n))


def tau_q(sigma: int, num: int, den: int, n: int) -> int:
    return int(lib().or_tau(sigma, num, den, n))


def hash64(seed: int, r: int) -> int:
    return int(lib().or_hash(seed, r))


def _pat(labels, edges):
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1), dtype=np.int32)
    if e.size == 0:
        e = np.zeros(2, dtype=np.int32)
        m = 0
    else:
        m = e.size // 2
    return lab, m, e


def canonical(labels, edges):
    """(labels in canonical order, code bits, perm) with labels used as given."""
    lab, m, e = _pat(labels, edges)
    n = lab.size
    ol = np.zeros(n, np.int32)
    op = np.zeros(n, np.int32)
    bits = C.c_uint32()
    if lib().or_canonical(n, lab, m, e, ol, C.byref(bits), op) != 0:
        raise ValueError("bad pattern")
    return tuple(int(x) for x in ol), int(bits.value), tuple(int(x) for x in op)


class Graph:
    """Oracle-side data graph.  Labels are arbitrary non-negative ids; seed fixes the greedy
    order (reading R4 in oracle.c)."""

    DEFAULT_SEED = 0x5EED

    def __init__(self, labels, src, dst, seed: int = DEFAULT_SEED, root_order: str = "hash",
                 directed: bool = False):
        self.labels = np.ascontiguousarray(labels, dtype=np.int32)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        if self.src.size == 0:
            self.src = np.zeros(1, np.int32)
            self.dst = np.zeros(1, np.int32)
            ne = 0
        else:
            ne = self.src.size
        self.nv = self.labels.size
        self.seed = seed
        self.directed = bool(directed)
        self._h = lib().or_graph_new2(self.nv, self.labels, ne, self.src, self.dst, seed, 1 if directed else 0)
        if root_order not in ("hash", "id"):
            raise ValueError(root_order)
        lib().or_graph_set_root_order(self._h, 1 if root_order == "id" else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_graph_free(h)
            self._h = None

    @property
    def arcs(self) -> int:
        return int(lib().or_graph_arcs(self._h))

    def rank(self, label: int) -> int:
        return int(lib().or_graph_rank(self._h, label))

    def support(self, labels, edges, sigma: int, lam: float = None, *, lam_num: int = None,
                lam_den: int = LAMBDA_DEN, mode: str = "early", tier: int = 1,
                want_selected: bool = False, budget: int = 0):
        """Support of one pattern.  Returns a dict with tau, mis, mni, n_maps (tier 0), frequent,
        and (optionally) the selected maps as canonical-vertex-indexed tuples.  mode "early",
        "early_nomni" (mni = -1) or "full".  budget > 0: None when the searches try more
        candidate vertices than that (the pattern is skipped)."""
        if lam_num is None:
            lam_num = lam_q(lam)
        lab, m, e = _pat(labels, edges)
        out = np.zeros(8, np.int64)
        sel_cap = 1 << 20 if want_selected else 0
        sel = np.zeros((max(sel_cap, 1), 8), np.int32)
        nsel = C.c_int64()
        mcode = {"full": 0, "early": 1, "early_nomni": 2}[mode]
        rc = lib().or_support_budget(self._h, lab.size, lab, m, e, sigma, lam_num, lam_den, mcode, tier, out,
                                     sel.ctypes.data if want_selected else None, sel_cap, C.byref(nsel), budget)
        if rc == -3:
            return None
        if rc != 0:
            raise ValueError("invalid pattern or parameters")
        res = dict(tau=int(out[0]), mis=int(out[1]), mni=int(out[2]),
                   n_maps=int(out[3]) if tier == 0 else None, frequent=bool(out[4]),
                   n=int(out[5]))
        if want_selected:
            res["selected"] = [tuple(int(x) for x in sel[i, : lab.size]) for i in range(nsel.value)]
        return res

    def count_maps(self, labels, edges, cap: int = 0) -> int:
        lab, m, e = _pat(labels, edges)
        return int(lib().or_count_maps(self._h, lab.size, lab, m, e, cap))

    def overlap_graph(self, labels, edges, max_maps: int = 1 << 20, cap_inst: int = 1 << 14,
                      cap_edges: int = 1 << 22):
        """(instances, conflict edges): instances = sorted list of sorted image vertex tuples,
        edges = sorted list of (a, b), a < b, instance indices whose vertex sets meet.  None if
        the maps or instances exceed the limits."""
        lab, m, e = _pat(labels, edges)
        n = lab.size
        inst = np.zeros((cap_inst, 8), np.int32)
        ed = np.zeros((cap_edges, 2), np.int32)
        ni, ne = C.c_int64(), C.c_int64()
        rc = lib().or_overlap_graph(self._h, n, lab, m, e, max_maps, inst.reshape(-1), cap_inst,
                                    C.byref(ni), ed.reshape(-1), cap_edges, C.byref(ne))
        if rc == -1:
            raise ValueError("bad pattern")
        if rc == -2:
            return None
        return ([tuple(int(x) for x in inst[i, :n]) for i in range(ni.value)],
                [(int(ed[i, 0]), int(ed[i, 1])) for i in range(ne.value)])

    def max_independent_set(self, labels, edges, max_maps: int = 1 << 20, max_inst: int = 64):
        """Size of a maximum independent set of the maps (Sec. 2.4.2), or None beyond the limits
        (the search is exhaustive)."""
        lab, m, e = _pat(labels, edges)
        r = int(lib().or_max_independent_set(self._h, lab.size, lab, m, e, max_maps, max_inst))
        if r == -1:
            raise ValueError("bad pattern")
        return None if r == -2 else r

    def mine(self, sigma: int, lam: float, max_edges: int):
        """Algorithm 1 with the predicate candidate generator.  Returns (patterns, levels) where
        patterns is a list of (n, rank labels tuple, bits, tau, mis, mni) sorted by
        (n, canonical code) and levels maps k -> (candidates, frequent)."""
        L = lib()
        h = L.or_mine(self._h, sigma, lam_q(lam), LAMBDA_DEN, max_edges)
        try:
            cnt = L.or_mined_count(h)
            out = []
            lab = np.zeros(8, np.int32)
            res = np.zeros(4, np.int64)
            n = C.c_int32()
            bits = C.c_uint32()
            for i in range(cnt):
                L.or_mined_get(h, i, C.byref(n), lab, C.byref(bits), res)
                out.append((n.value, tuple(int(x) for x in lab[: n.value]), int(bits.value),
                            int(res[0]), int(res[1]), int(res[2])))
            cand = np.zeros(9, np.int64)
            freq = np.zeros(9, np.int64)
            L.or_mined_levels(h, cand, freq)
            levels = {k: (int(cand[k]), int(freq[k])) for k in range(2, 9) if cand[k] > 0}
            return out, levels
        finally:
            L.or_mined_free(h)


def candidates(patterns, max_edges: int = 0):
    """Candidate k-vertex patterns from a list of frequent (k-1)-vertex patterns given as
    (labels, edges).  Returns sorted canonical codes (n, labels tuple, bits)."""
    cnt = len(patterns)
    ns = np.zeros(max(cnt, 1), np.int32)
    ms = np.zeros(max(cnt, 1), np.int32)
    lab = np.zeros((max(cnt, 1), 8), np.int32)
    edg = np.zeros((max(cnt, 1), 56), np.int32)
    for i, (l, e) in enumerate(patterns):
        l = np.asarray(l, np.int32)
        e = np.asarray(e, np.int32).reshape(-1)
        ns[i] = l.size
        ms[i] = e.size // 2
        lab[i, : l.size] = l
        edg[i, : e.size] = e
    cap = 1 << 16
    on = np.zeros(cap, np.int32)
    ol = np.zeros(cap * 8, np.int32)
    ob = np.zeros(cap, np.uint32)
    k = lib().or_candidates(cnt, ns, lab.reshape(-1), ms, edg.reshape(-1), max_edges, on, ol, ob, cap)
    if k < 0:
        raise RuntimeError("too many candidates")
    return [(int(on[i]), tuple(int(x) for x in ol[8 * i: 8 * i + on[i]]), int(ob[i])) for i in range(k)]
