"""Python binding of libflexis.so (the C ABI in include/flexis.h).

Argument marshalling only: every step of support evaluation runs in the library's CUDA kernels
and host runtime.  There is no fallback: if the compiled library is missing, importing the
binding's entry points raises.

Function names follow the C ABI (flexis_load_graph, flexis_support, flexis_support_batch,
flexis_mine, flexis_serve_*, ...); `Graph` and `Server` wrap the handles.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libflexis.so")

FLEXIS_OK = 0
FLEXIS_E_INVALID = -1
FLEXIS_E_NOMEM = -2
FLEXIS_E_CUDA = -3
FLEXIS_E_TIMEOUT = -4
FLEXIS_E_CANCELLED = -5
FLEXIS_E_UNSUPPORTED = -6
FLEXIS_E_BUSY = -7
FLEXIS_MODE_FULL = 0
FLEXIS_MODE_EARLY = 1
FLEXIS_MODE_NO_MNI = 4
FLEXIS_MODE_COUNT_MAPS = 8
FLEXIS_MODE_NO_MIS = 16
FLEXIS_MODE_EXACT_MIS = 32
FLEXIS_FLAG_ABSENT_LABEL = 1
FLEXIS_FLAG_MNI_FROM_MIS = 2
FLEXIS_FLAG_MNI_SKIPPED = 4
FLEXIS_FLAG_MIS_SATURATED = 8
FLEXIS_FLAG_MNI_SATURATED = 16
FLEXIS_FLAG_MAPS_SATURATED = 32
FLEXIS_FLAG_MIS_SKIPPED = 64
FLEXIS_FLAG_EXACT_MIS_SATURATED = 128
FLEXIS_LAYOUT_VREC = 0
FLEXIS_LAYOUT_RUNS = 1
FLEXIS_LAYOUT_ADJ = 2
FLEXIS_LAYOUT_LAB_VTX = 3
LAMBDA_DEN = 1_000_000
DEFAULT_SEED = 0x5EED


class FlexisError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


class flexis_options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("device", C.c_int32), ("window_min", C.c_int32),
                ("window_max", C.c_int32), ("search_blocks", C.c_int32),
                ("record_selected", C.c_int32), ("search_budget", C.c_int32),
                ("split_pieces", C.c_int32), ("sub_searches", C.c_int32), ("timing", C.c_int32),
                ("graphs", C.c_int32), ("deadline_ms", C.c_int32), ("root_order", C.c_int32),
                ("directed", C.c_int32), ("maps_cap", C.c_int64),
                ("frontier_rows", C.c_int64), ("exact_mis_nodes", C.c_int64),
                ("exact_mis_maps", C.c_int32), ("autotune", C.c_int32), ("host_build", C.c_int32),
                ("reserved", C.c_int32 * 4)]


class flexis_pattern(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("labels", C.POINTER(C.c_int32)),
                ("edges", C.POINTER(C.c_int32)), ("edge_labels", C.POINTER(C.c_int32))]


class flexis_support_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n", C.c_int32), ("sigma", C.c_int64), ("tau", C.c_int64),
                ("cap", C.c_int64), ("mis", C.c_int64), ("mni", C.c_int64),
                ("frequent", C.c_int32), ("flags", C.c_uint32), ("n_maps", C.c_uint64),
                ("mis_exact", C.c_int64), ("roots_searched", C.c_int64),
                ("search_steps", C.c_int64), ("max_item_steps", C.c_int32), ("rounds", C.c_int32)]

    def as_dict(self):
        return dict(status=self.status, n=self.n, sigma=self.sigma, tau=self.tau, cap=self.cap,
                    mis=self.mis, mni=self.mni, frequent=bool(self.frequent), flags=self.flags,
                    n_maps=self.n_maps, mis_exact=self.mis_exact,
                    roots_searched=self.roots_searched, search_steps=self.search_steps,
                    max_item_steps=self.max_item_steps, rounds=self.rounds)


RESULT_DTYPE = np.dtype([("status", "<i4"), ("n", "<i4"), ("sigma", "<i8"), ("tau", "<i8"),
                         ("cap", "<i8"), ("mis", "<i8"), ("mni", "<i8"), ("frequent", "<i4"),
                         ("flags", "<u4"), ("n_maps", "<u8"), ("mis_exact", "<i8"), ("roots", "<i8"),
                         ("steps", "<i8"), ("maxsteps", "<i4"), ("rounds", "<i4")])


class flexis_plan(C.Structure):
    _fields_ = [("bytes", C.c_uint8 * 1024)]


class flexis_graph_info(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("n_arcs", C.c_int64), ("n_self_loops", C.c_int64),
                ("n_duplicates", C.c_int64), ("n_labels", C.c_int32), ("max_degree", C.c_int32),
                ("device_bytes", C.c_int64), ("sm_count", C.c_int32), ("l2_bytes", C.c_int32),
                ("n_input_vertices", C.c_int64), ("edge_label_base", C.c_int32), ("directed", C.c_int32),
                ("built_on_device", C.c_int32), ("upload_bytes", C.c_int64)]


class flexis_stats(C.Structure):
    _fields_ = [("rounds", C.c_int64), ("search_items", C.c_int64), ("mni_items", C.c_int64),
                ("kernel_launches", C.c_int64), ("alg_bytes", C.c_int64),
                ("alg_bytes_greedy", C.c_int64), ("patterns", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("search_ms", C.c_float), ("mni_ms", C.c_float),
                ("total_ms", C.c_float), ("host_gen_ms", C.c_float), ("host_compile_ms", C.c_float),
                ("search_launches", C.c_int32), ("batches", C.c_int32), ("graph_launches", C.c_int32),
                ("enum_rows", C.c_int64), ("enum_scanned", C.c_int64), ("enum_bytes", C.c_int64),
                ("search_scanned", C.c_int64), ("search_bound", C.c_int64), ("search_map_words", C.c_int64),
                ("autotune_probes", C.c_int32), ("search_budget", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# symbol table: name -> (restype, argtypes); every symbol include/flexis.h declares
_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)
_I64P = C.POINTER(C.c_int64)
SYMBOLS = {
    "flexis_status_string": (C.c_char_p, [C.c_int]),
    "flexis_default_options": (None, [C.POINTER(flexis_options)]),
    "flexis_lambda_quantize": (C.c_int, [C.c_double, _I64P]),
    "flexis_load_graph": (C.c_int, [C.c_int64, _I32P, C.c_int64, _I32P, _I32P,
                                     C.POINTER(flexis_options), C.POINTER(_P)]),
    "flexis_load_graph_edge_labels": (C.c_int, [C.c_int64, _I32P, C.c_int64, _I32P, _I32P, _I32P,
                                                 C.POINTER(flexis_options), C.POINTER(_P)]),
    "flexis_free_graph": (None, [_P]),
    "flexis_graph_info_get": (C.c_int, [_P, C.POINTER(flexis_graph_info)]),
    "flexis_graph_layout": (C.c_int, [_P, C.c_int32, _P, C.c_int64, _I64P]),
    "flexis_support": (C.c_int, [_P, C.POINTER(flexis_pattern), C.c_int64, C.c_double, C.c_int32,
                                  C.POINTER(flexis_support_result)]),
    "flexis_support_q": (C.c_int, [_P, C.POINTER(flexis_pattern), C.c_int64, C.c_int64, C.c_int64,
                                    C.c_int32, C.POINTER(flexis_support_result)]),
    "flexis_support_batch": (C.c_int, [_P, C.POINTER(flexis_pattern), _I64P, C.POINTER(C.c_double),
                                        C.c_int32, C.c_int32, C.POINTER(flexis_support_result)]),
    "flexis_compile": (C.c_int, [_P, C.POINTER(flexis_pattern), _I64P, _I64P, C.c_int64, C.c_int32,
                                  C.c_int32, C.POINTER(flexis_plan)]),
    "flexis_support_plans_device": (C.c_int, [_P, _P, C.c_int32, _P, _P]),
    "flexis_last_stats": (C.c_int, [_P, C.POINTER(flexis_stats)]),
    "flexis_graph_stream": (C.c_void_p, [_P]),
    "flexis_support_noalloc": (C.c_int, [_P, C.POINTER(flexis_plan), C.POINTER(flexis_support_result), _P]),
    "flexis_selected_maps": (C.c_int, [_P, C.c_int32, _I32P, C.c_int64, _I64P]),
    "flexis_overlap_graph": (C.c_int, [_P, C.POINTER(flexis_pattern), _I32P, C.c_int64, _I64P, _I32P,
                                        C.c_int64, _I64P]),
    "flexis_mine": (C.c_int, [_P, C.c_int64, C.c_double, C.c_int32, C.POINTER(_P)]),
    "flexis_pattern_set_count": (C.c_int64, [_P]),
    "flexis_pattern_set_get": (C.c_int, [_P, C.c_int64, _I32P, _I32P, _I32P, _I32P, _I32P,
                                          C.POINTER(C.c_uint32), C.POINTER(flexis_support_result)]),
    "flexis_pattern_set_levels": (C.c_int, [_P, _I64P, _I64P]),
    "flexis_pattern_set_read": (C.c_int64, [_P, C.c_int64, C.c_int64, _I32P, _I32P,
                                            C.POINTER(C.c_uint32), _I32P,
                                            C.POINTER(flexis_support_result)]),
    "flexis_free_pattern_set": (None, [_P]),
    "flexis_canonical_code": (C.c_int, [C.POINTER(flexis_pattern), _I32P, C.POINTER(C.c_uint32), _I32P]),
    "flexis_generate_candidates": (C.c_int64, [C.POINTER(flexis_pattern), C.c_int32, C.c_int32, _I32P,
                                               _I32P, C.POINTER(C.c_uint32), C.c_int64]),
    "flexis_serve_start": (C.c_int, [_P, C.c_int32, C.POINTER(_P)]),
    "flexis_serve_submit": (C.c_int, [_P, C.c_int64, C.POINTER(flexis_pattern), C.c_int64,
                                       C.c_double, C.c_int32]),
    "flexis_serve_poll": (C.c_int, [_P, _I64P, C.POINTER(flexis_support_result),
                                     C.POINTER(C.c_double), C.c_int32, _I32P]),
    "flexis_serve_stop": (C.c_int, [_P]),
}

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libflexis.so.  Raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libflexis.so is not built ({LIB_PATH}); run "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SYMBOLS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def lambda_quantize(lam: float) -> int:
    """Numerator of lambda over LAMBDA_DEN, as the library quantises it (flexis_lambda_quantize)."""
    q = C.c_int64()
    _check(lib().flexis_lambda_quantize(float(lam), C.byref(q)), "flexis_lambda_quantize")
    return int(q.value)


def status_string(code: int) -> str:
    try:
        return lib().flexis_status_string(code).decode()
    except Exception:
        return "unknown"


def _check(code, what):
    if code != FLEXIS_OK:
        raise FlexisError(code, what)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def make_pattern(labels, edges, edge_labels=None):
    """(flexis_pattern, keepalive) from label list, edge list and (edge-labelled graphs) the
    edges' labels."""
    lab = _i32(labels)
    e = _i32(np.asarray(edges, dtype=np.int32).reshape(-1)) if len(edges) else np.zeros(2, np.int32)
    m = (e.size // 2) if len(edges) else 0
    el = None if edge_labels is None else _i32(edge_labels)
    p = flexis_pattern(lab.size, m, lab.ctypes.data_as(_I32P), e.ctypes.data_as(_I32P),
                       el.ctypes.data_as(_I32P) if el is not None else None)
    return p, (lab, e, el)


def default_options(**kw) -> flexis_options:
    o = flexis_options()
    lib().flexis_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


class Graph:
    """A data graph resident on one GPU (flexis_load_graph).

    Keyword options are the fields of flexis_options: seed, device, window_min, window_max,
    search_blocks, record_selected, search_budget, split_pieces, sub_searches, timing, graphs,
    deadline_ms, root_order, directed, maps_cap, frontier_rows, exact_mis_nodes,
    exact_mis_maps, autotune, host_build (meanings in include/flexis.h).  They apply to every
    call on the graph and to servers started on it."""

    def __init__(self, labels, src, dst, edge_labels=None, **options):
        L = lib()
        self._labels = _i32(labels)
        self._src = _i32(src)
        self._dst = _i32(dst)
        self.options = default_options(**options)
        h = _P()
        ne = self._src.size
        srcp = self._src if ne else np.zeros(1, np.int32)
        dstp = self._dst if ne else np.zeros(1, np.int32)
        if edge_labels is None:
            rc = L.flexis_load_graph(self._labels.size, self._labels.ctypes.data_as(_I32P), ne,
                                     srcp.ctypes.data_as(_I32P), dstp.ctypes.data_as(_I32P),
                                     C.byref(self.options), C.byref(h))
            _check(rc, "flexis_load_graph")
        else:
            el = _i32(edge_labels)
            elp = el if ne else np.zeros(1, np.int32)
            rc = L.flexis_load_graph_edge_labels(self._labels.size, self._labels.ctypes.data_as(_I32P), ne,
                                                 srcp.ctypes.data_as(_I32P), dstp.ctypes.data_as(_I32P),
                                                 elp.ctypes.data_as(_I32P), C.byref(self.options), C.byref(h))
            _check(rc, "flexis_load_graph_edge_labels")
        self._h = h
        del self._src, self._dst

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().flexis_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = flexis_graph_info()
        _check(lib().flexis_graph_info_get(self._h, C.byref(i)), "flexis_graph_info_get")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def layout(self, part: int) -> np.ndarray:
        """One resident layout array (flexis_graph_layout): FLEXIS_LAYOUT_VREC as uint32 rows of
        8 words, the others as flat uint32 / int32 arrays."""
        n = C.c_int64()
        _check(lib().flexis_graph_layout(self._h, part, None, 0, C.byref(n)), "flexis_graph_layout")
        dt = np.uint32 if part in (FLEXIS_LAYOUT_VREC, FLEXIS_LAYOUT_RUNS) else np.int32
        out = np.zeros(n.value // 4, dtype=dt)
        _check(lib().flexis_graph_layout(self._h, part, out.ctypes.data_as(_P), n.value, C.byref(n)),
               "flexis_graph_layout")
        return out.reshape(-1, 8) if part == FLEXIS_LAYOUT_VREC else out

    def support(self, labels, edges, sigma, lam=None, *, lam_num=None, lam_den=LAMBDA_DEN,
                mode=FLEXIS_MODE_EARLY, edge_labels=None) -> dict:
        p, keep = make_pattern(labels, edges, edge_labels)
        r = flexis_support_result()
        if lam_num is not None:
            rc = lib().flexis_support_q(self._h, C.byref(p), sigma, lam_num, lam_den, mode, C.byref(r))
        else:
            rc = lib().flexis_support(self._h, C.byref(p), sigma, float(lam), mode, C.byref(r))
        _check(rc, "flexis_support")
        return r.as_dict()

    def _patterns(self, patterns):
        arr = (flexis_pattern * max(1, len(patterns)))()
        keep = []
        for i, pt in enumerate(patterns):  # (labels, edges) or (labels, edges, edge_labels)
            p, k = make_pattern(*pt)
            arr[i] = p
            keep.append(k)
        return arr, keep

    def support_batch(self, patterns, sigma, lam, mode=FLEXIS_MODE_EARLY) -> list[dict]:
        cnt = len(patterns)
        arr, keep = self._patterns(patterns)
        sig = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, np.int64), (cnt,)))
        lm = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (cnt,)))
        out = (flexis_support_result * max(1, cnt))()
        rc = lib().flexis_support_batch(self._h, arr, sig.ctypes.data_as(_I64P),
                                        lm.ctypes.data_as(C.POINTER(C.c_double)), cnt, mode, out)
        _check(rc, "flexis_support_batch")
        return [out[i].as_dict() for i in range(cnt)]

    def compile(self, patterns, sigma, lam, mode=FLEXIS_MODE_EARLY) -> np.ndarray:
        """Plans (uint8 [count, 1024]) of the patterns, ready to be copied to device memory."""
        cnt = len(patterns)
        arr, keep = self._patterns(patterns)
        sig = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, np.int64), (cnt,)))
        lams = np.broadcast_to(np.asarray(lam, np.float64), (cnt,))
        num = np.zeros(max(cnt, 1), np.int64)
        for i in range(cnt):
            num[i] = lambda_quantize(float(lams[i]))
        plans = np.zeros((max(1, cnt), 1024), np.uint8)
        rc = lib().flexis_compile(self._h, arr, sig.ctypes.data_as(_I64P), num.ctypes.data_as(_I64P),
                                  LAMBDA_DEN, cnt, mode, plans.ctypes.data_as(C.POINTER(flexis_plan)))
        _check(rc, "flexis_compile")
        return plans[:cnt]

    def support_plans_device(self, d_plans_ptr: int, count: int, d_results_ptr: int, stream_ptr: int = 0):
        rc = lib().flexis_support_plans_device(self._h, C.c_void_p(d_plans_ptr), count,
                                               C.c_void_p(d_results_ptr), C.c_void_p(stream_ptr))
        _check(rc, "flexis_support_plans_device")

    def support_noalloc(self, plan: np.ndarray, stream: int = 0) -> dict:
        """flexis_support_noalloc on one compiled plan (a uint8[1024] row of compile())."""
        buf = np.ascontiguousarray(plan, dtype=np.uint8).reshape(-1)
        if buf.size != C.sizeof(flexis_plan):
            raise ValueError("one plan of %d bytes expected" % C.sizeof(flexis_plan))
        r = flexis_support_result()
        _check(lib().flexis_support_noalloc(self._h, buf.ctypes.data_as(C.POINTER(flexis_plan)),
                                            C.byref(r), C.c_void_p(stream)), "flexis_support_noalloc")
        return r.as_dict()

    def stream(self) -> int:
        """cudaStream_t (as an int) on which this graph's evaluations run."""
        return int(lib().flexis_graph_stream(self._h) or 0)

    def stats(self) -> dict:
        s = flexis_stats()
        _check(lib().flexis_last_stats(self._h, C.byref(s)), "flexis_last_stats")
        return s.as_dict()

    def selected_maps(self, i: int, n: int, cap: int = 1 << 20):
        buf = np.zeros((cap, 8), np.int32)
        k = C.c_int64()
        _check(lib().flexis_selected_maps(self._h, i, buf.ctypes.data_as(_I32P), cap, C.byref(k)),
               "flexis_selected_maps")
        return [tuple(int(x) for x in buf[j, :n]) for j in range(k.value)]

    def overlap_graph(self, labels, edges, cap_instances=1 << 12, cap_edges=1 << 22, edge_labels=None):
        """flexis_overlap_graph: (instances, conflict edges), instances as sorted vertex tuples
        in ascending order, edges as (a, b) pairs, a < b, ascending."""
        p, keep = make_pattern(labels, edges, edge_labels)
        inst = np.zeros((max(cap_instances, 1), 8), np.int32)
        ed = np.zeros((max(cap_edges, 1), 2), np.int32)
        ni, ne = C.c_int64(), C.c_int64()
        _check(lib().flexis_overlap_graph(self._h, C.byref(p), inst.ctypes.data_as(_I32P), cap_instances,
                                          C.byref(ni), ed.ctypes.data_as(_I32P), cap_edges, C.byref(ne)),
               "flexis_overlap_graph")
        n = p.n
        k = min(ni.value, cap_instances)
        return ([tuple(int(x) for x in inst[i, :n]) for i in range(k)],
                [(int(ed[i, 0]), int(ed[i, 1])) for i in range(min(ne.value, cap_edges))])

    def mine(self, sigma, lam, max_edges):
        """Algorithm 1.  Returns (patterns, levels): patterns = list of dict(n, labels, edges,
        code_labels, code_bits, tau, mis, mni) sorted by (n, canonical code); levels maps
        k -> (candidates, frequent)."""
        arr, levels = self.mine_arrays(sigma, lam, max_edges)
        out = []
        for i in range(arr["n"].size):
            n = int(arr["n"][i])
            bits = int(arr["code_bits"][i])
            # edges of the canonical pattern from its code bits (column j, rows i < j; bit set =
            # not adjacent; first bit most significant)
            edges, t = [], n * (n - 1) // 2 - 1
            for b in range(1, n):
                for a in range(b):
                    if not (bits >> t) & 1:
                        edges.append((a, b))
                    t -= 1
            out.append(dict(n=n, labels=tuple(int(x) for x in arr["labels"][i, :n]), edges=edges,
                            code_labels=tuple(int(x) for x in arr["code_labels"][i, :n]), code_bits=bits,
                            tau=int(arr["tau"][i]), mis=int(arr["mis"][i]), mni=int(arr["mni"][i]),
                            frequent=True))
        return out, levels

    def mine_arrays(self, sigma, lam, max_edges):
        """Algorithm 1 with the frequent set read back in one call: (dict of numpy arrays n,
        code_labels, code_bits, labels, tau, mis, mni; levels)."""
        L = lib()
        h = _P()
        _check(L.flexis_mine(self._h, sigma, float(lam), max_edges, C.byref(h)), "flexis_mine")
        try:
            cnt = int(L.flexis_pattern_set_count(h))
            n = np.zeros(max(cnt, 1), np.int32)
            clab = np.zeros((max(cnt, 1), 8), np.int32)
            lab = np.zeros((max(cnt, 1), 8), np.int32)
            bits = np.zeros(max(cnt, 1), np.uint32)
            res = (flexis_support_result * max(cnt, 1))()
            got = L.flexis_pattern_set_read(h, 0, cnt, n.ctypes.data_as(_I32P), clab.ctypes.data_as(_I32P),
                                            bits.ctypes.data_as(C.POINTER(C.c_uint32)),
                                            lab.ctypes.data_as(_I32P), res)
            if got != cnt:
                raise FlexisError(FLEXIS_E_INVALID, "flexis_pattern_set_read")
            rr = np.frombuffer(res, dtype=RESULT_DTYPE, count=cnt)
            cand = np.zeros(9, np.int64)
            freq = np.zeros(9, np.int64)
            L.flexis_pattern_set_levels(h, cand.ctypes.data_as(_I64P), freq.ctypes.data_as(_I64P))
            levels = {k: (int(cand[k]), int(freq[k])) for k in range(2, 9) if cand[k] > 0}
            arr = dict(n=n[:cnt], code_labels=clab[:cnt], code_bits=bits[:cnt], labels=lab[:cnt],
                       tau=rr["tau"].copy(), mis=rr["mis"].copy(), mni=rr["mni"].copy())
            return arr, levels
        finally:
            L.flexis_free_pattern_set(h)


def canonical_code(labels, edges):
    p, keep = make_pattern(labels, edges)
    n = p.n
    lab = np.zeros(max(n, 1), np.int32)
    perm = np.zeros(max(n, 1), np.int32)
    bits = C.c_uint32()
    _check(lib().flexis_canonical_code(C.byref(p), lab.ctypes.data_as(_I32P), C.byref(bits),
                                       perm.ctypes.data_as(_I32P)), "flexis_canonical_code")
    return tuple(int(x) for x in lab[:n]), int(bits.value), tuple(int(x) for x in perm[:n])


def generate_candidates(patterns, max_edges=0):
    arr = (flexis_pattern * max(1, len(patterns)))()
    keep = []
    for i, pt in enumerate(patterns):
        p, k = make_pattern(*pt)
        arr[i] = p
        keep.append(k)
    cap = 1 << 18
    while True:
        on = np.zeros(cap, np.int32)
        ol = np.zeros(cap * 8, np.int32)
        ob = np.zeros(cap, np.uint32)
        k = lib().flexis_generate_candidates(arr, len(patterns), max_edges, on.ctypes.data_as(_I32P),
                                             ol.ctypes.data_as(_I32P),
                                             ob.ctypes.data_as(C.POINTER(C.c_uint32)), cap)
        if k == FLEXIS_E_INVALID:
            raise FlexisError(FLEXIS_E_INVALID, "flexis_generate_candidates")
        if k >= 0:
            break
        cap = -k  # the output needs -k entries
    return [(int(on[i]), tuple(int(x) for x in ol[8 * i: 8 * i + on[i]]), int(ob[i])) for i in range(k)]


class Server:
    """Continuous-batching support server on a resident graph (flexis_serve_*)."""

    def __init__(self, graph: Graph, slots: int = 0):
        h = _P()
        _check(lib().flexis_serve_start(graph.handle, slots, C.byref(h)), "flexis_serve_start")
        self._h = h
        self.graph = graph

    def submit(self, request_id, labels, edges, sigma, lam, mode=FLEXIS_MODE_EARLY, edge_labels=None):
        p, keep = make_pattern(labels, edges, edge_labels)
        return lib().flexis_serve_submit(self._h, request_id, C.byref(p), sigma, float(lam), mode)

    def poll(self, max_results=4096):
        ids = np.zeros(max_results, np.int64)
        res = (flexis_support_result * max_results)()
        lat = np.zeros(max_results, np.float64)
        n = C.c_int32()
        rc = lib().flexis_serve_poll(self._h, ids.ctypes.data_as(_I64P), res,
                                     lat.ctypes.data_as(C.POINTER(C.c_double)), max_results, C.byref(n))
        _check(rc, "flexis_serve_poll")
        return [(int(ids[i]), res[i].as_dict(), float(lat[i])) for i in range(n.value)]

    def stop(self):
        if getattr(self, "_h", None):
            rc = lib().flexis_serve_stop(self._h)
            self._h = None
            _check(rc, "flexis_serve_stop")
