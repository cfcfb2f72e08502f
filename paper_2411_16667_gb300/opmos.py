"""ctypes binding of the C ABI in include/opmos.h (argument marshalling only).

Every function here forwards to the CUDA library; none computes any part of
the search. Loading fails loudly (``OpmosError``) when ``libopmos.so`` has not
been built -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from collections.abc import Sequence

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libopmos.so")
_lib = None

OK, ERR_INVALID_ARG, ERR_OVERFLOW, ERR_OUT_OF_MEMORY, ERR_CAPACITY, ERR_BUDGET, ERR_TIMEOUT, ERR_CUDA, PENDING = range(9)
FLAG_NO_PATHS = 1
FLAG_GRAPH = 2
FLAG_FIFO = 4
MAX_D = 16

TEST_EXPORTS = ("opmos_test_merge", "opmos_test_window")  # include/opmos_test.h
EXPORTS = ("opmos_default_options", "opmos_device_count", "opmos_graph_create", "opmos_graph_destroy",
           "opmos_heuristic", "opmos_heuristic_copy", "opmos_heuristic_destroy", "opmos_solve",
           "opmos_solve_batch", "opmos_result_count", "opmos_result_d", "opmos_result_costs",
           "opmos_result_path", "opmos_result_stats", "opmos_result_free", "opmos_server_create",
           "opmos_server_submit", "opmos_server_poll", "opmos_server_destroy", "opmos_last_error",
           "opmos_heuristic_noalloc", "opmos_result_paths")


class OpmosError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"opmos error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("window", ctypes.c_uint32), ("lanes_per_label", ctypes.c_uint32), ("tile", ctypes.c_uint32),
                ("delta", ctypes.c_uint32), ("label_budget", ctypes.c_uint64),
                ("mem_budget_bytes", ctypes.c_uint64), ("d_used", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("alone_labels", ctypes.c_uint64), ("alone_window", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("stream", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in (
        "extracted", "dead_skipped", "goal_pruned", "candidates", "inserted", "pruned", "steps",
        "frontier_cmp", "p_cmp", "bytes", "heuristic_ns", "search_ns", "total_ns")] + [
        ("phase_ns", ctypes.c_uint64 * 4), ("goal_inserted", ctypes.c_uint64),
        ("open_scanned", ctypes.c_uint64), ("open_rewritten", ctypes.c_uint64),
        ("list_candidates", ctypes.c_uint64), ("longest_task_ns", ctypes.c_uint64 * 3),
        ("heavy_merges", ctypes.c_uint64), ("heavy_max_candidates", ctypes.c_uint64),
        ("heavy_max_frontier", ctypes.c_uint64), ("task_ns", ctypes.c_uint64 * 3)]

    def as_dict(self) -> dict:
        arrays = ("phase_ns", "longest_task_ns", "task_ns")
        d = {f: int(getattr(self, f)) for f, _ in self._fields_ if f not in arrays}
        for f in arrays:
            d[f] = [int(x) for x in getattr(self, f)]
        return d


def lib(path: str | None = None):
    """Load the CUDA library (raises OpmosError if it is not built)."""
    global _lib
    if _lib is None:
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise OpmosError(ERR_CUDA, f"{p} is not built; run paper_2411_16667_gb300.build()")
        L = ctypes.CDLL(p)
        u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
        pp = ctypes.POINTER(vp)
        L.opmos_default_options.argtypes = [ctypes.POINTER(Options)]
        L.opmos_default_options.restype = None
        L.opmos_device_count.restype = ctypes.c_int
        L.opmos_graph_create.argtypes = [u32, u64, u32, vp, vp, vp, pp]
        L.opmos_graph_destroy.argtypes = [vp]
        L.opmos_graph_destroy.restype = None
        L.opmos_heuristic.argtypes = [vp, u32, u32, pp]
        L.opmos_heuristic_copy.argtypes = [vp, vp]
        L.opmos_heuristic_destroy.argtypes = [vp]
        L.opmos_heuristic_destroy.restype = None
        L.opmos_solve.argtypes = [vp, vp, u32, u32, ctypes.POINTER(Options), pp]
        L.opmos_solve_batch.argtypes = [vp, u32, vp, vp, ctypes.POINTER(Options), vp, vp]
        L.opmos_result_count.argtypes = [vp]
        L.opmos_result_count.restype = u32
        L.opmos_result_d.argtypes = [vp]
        L.opmos_result_d.restype = u32
        L.opmos_result_costs.argtypes = [vp, vp]
        L.opmos_result_path.argtypes = [vp, u32, vp, vp, u32, ctypes.POINTER(u32)]
        L.opmos_result_paths.argtypes = [vp, vp, vp, vp]
        L.opmos_result_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.opmos_result_free.argtypes = [vp]
        L.opmos_result_free.restype = None
        L.opmos_server_create.argtypes = [vp, u32, ctypes.POINTER(Options), pp]
        L.opmos_server_submit.argtypes = [vp, u32, u32, u32, u32, ctypes.POINTER(u64)]
        L.opmos_server_poll.argtypes = [vp, u64, pp]
        L.opmos_server_destroy.argtypes = [vp]
        L.opmos_server_destroy.restype = None
        L.opmos_last_error.restype = ctypes.c_char_p
        L.opmos_heuristic_noalloc.argtypes = [vp, u32, u32, vp, vp]
        L.opmos_test_merge.argtypes = [u32, u32, vp, u32, vp, vp, u32, u32, u32, vp, vp, ctypes.POINTER(u32)]
        L.opmos_test_window.argtypes = [u32, vp, vp, vp, u32, vp, vp, ctypes.POINTER(u32)]
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        msg = lib().opmos_last_error().decode(errors="replace")
        raise OpmosError(rc, f"{what}: {msg}")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def opmos_default_options(**kw) -> Options:
    o = Options()
    lib().opmos_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def opmos_device_count() -> int:
    return int(lib().opmos_device_count())


class opmos_graph:
    """Device-resident graph (opmos_graph_create / opmos_graph_destroy)."""

    def __init__(self, n: int, d: int, rowptr, col, cost):
        self.rowptr = np.ascontiguousarray(rowptr, np.uint64)
        self.col = np.ascontiguousarray(col, np.uint32)
        self.cost = np.ascontiguousarray(cost, np.uint32).reshape(-1)
        self.n, self.d, self.m = int(n), int(d), int(self.col.shape[0])
        h = ctypes.c_void_p()
        _check(lib().opmos_graph_create(self.n, self.m, self.d, _ptr(self.rowptr), _ptr(self.col),
                                        _ptr(self.cost), ctypes.byref(h)), "opmos_graph_create")
        self.handle = h

    @classmethod
    def from_synth(cls, g) -> "opmos_graph":
        return cls(g.n, g.d, g.rowptr, g.col, g.cost)

    def close(self):
        if getattr(self, "handle", None):
            lib().opmos_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class opmos_heur:
    """Device-resident ideal-point heuristic (opmos_heuristic)."""

    def __init__(self, graph: opmos_graph, goal: int, d_used: int = 0):
        h = ctypes.c_void_p()
        _check(lib().opmos_heuristic(graph.handle, goal, d_used, ctypes.byref(h)), "opmos_heuristic")
        self.handle, self.graph, self.goal = h, graph, goal
        self.d = d_used or graph.d

    def copy(self) -> np.ndarray:
        out = np.empty((self.d, self.graph.n), np.uint32)
        _check(lib().opmos_heuristic_copy(self.handle, _ptr(out)), "opmos_heuristic_copy")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().opmos_heuristic_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def opmos_heuristic_noalloc(graph: opmos_graph, goal: int, d_used: int, h_out_device_ptr: int,
                            stream_ptr: int | None = None) -> None:
    """Heuristic into a caller-owned device buffer; allocates nothing on the device."""
    _check(lib().opmos_heuristic_noalloc(graph.handle, goal, d_used, ctypes.c_void_p(h_out_device_ptr),
                                         ctypes.c_void_p(stream_ptr) if stream_ptr else None),
           "opmos_heuristic_noalloc")


@dataclasses.dataclass
class Result:
    costs: np.ndarray  # uint32 [count, d], lexicographic
    paths: "Paths | None"  # paths[i] = (nodes uint32, edges uint64), or None
    stats: dict


class Paths(Sequence):
    """The paths of a result, one per cost vector, over three flat arrays
    (``opmos_result_paths``): ``paths[i]`` is (nodes, arc ids), views of
    ``nodes[offsets[i]:offsets[i+1]]`` and ``edges[offsets[i]-i:offsets[i+1]-i-1]``."""

    def __init__(self, offsets: np.ndarray, nodes: np.ndarray, edges: np.ndarray):
        self.offsets, self.nodes, self.edges = offsets, nodes, edges

    def __len__(self) -> int:
        return int(self.offsets.shape[0]) - 1

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(len(self)))]
        n = len(self)
        if i < 0:
            i += n
        if not 0 <= i < n:
            raise IndexError(i)
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return self.nodes[a:b], self.edges[a - i:b - i - 1]


def _take(res) -> Result:
    L = lib()
    try:
        cnt, d = L.opmos_result_count(res), L.opmos_result_d(res)
        costs = np.empty((cnt, d), np.uint32)
        if cnt:
            _check(L.opmos_result_costs(res, _ptr(costs)), "opmos_result_costs")
        st = Stats()
        _check(L.opmos_result_stats(res, ctypes.byref(st)), "opmos_result_stats")
        offs = np.zeros(cnt + 1, np.uint32)
        paths = None
        if L.opmos_result_paths(res, _ptr(offs), None, None) == OK:
            total = int(offs[cnt])
            nodes = np.empty(max(total, 1), np.uint32)
            edges = np.empty(max(total - cnt, 1), np.uint64)
            _check(L.opmos_result_paths(res, _ptr(offs), _ptr(nodes), _ptr(edges)), "opmos_result_paths")
            paths = Paths(offs, nodes[:total], edges[:total - cnt])
        return Result(costs, paths, st.as_dict())
    finally:
        L.opmos_result_free(res)


def _options(**kw) -> Options:
    """Options with only the given fields set; zero fields take the library
    default of the call they are passed to (single query or batch)."""
    o = Options()
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def opmos_solve(graph: opmos_graph, start: int, goal: int, heur: opmos_heur | None = None,
                options: Options | None = None, **kw) -> Result:
    o = options or _options(**kw)
    res = ctypes.c_void_p()
    _check(lib().opmos_solve(graph.handle, heur.handle if heur else None, start, goal, ctypes.byref(o),
                             ctypes.byref(res)), "opmos_solve")
    return _take(res)


def opmos_solve_batch(graph: opmos_graph, starts, goals, options: Options | None = None, **kw):
    """Returns a list of (status, Result or None)."""
    starts = np.ascontiguousarray(starts, np.uint32)
    goals = np.ascontiguousarray(goals, np.uint32)
    nq = int(starts.shape[0])
    o = options or _options(**kw)
    outs = (ctypes.c_void_p * max(nq, 1))()
    status = np.zeros(max(nq, 1), np.int32)
    _check(lib().opmos_solve_batch(graph.handle, nq, _ptr(starts), _ptr(goals), ctypes.byref(o),
                                   ctypes.cast(outs, ctypes.c_void_p), _ptr(status)), "opmos_solve_batch")
    results = []
    for q in range(nq):
        r = outs[q]
        results.append((int(status[q]), _take(ctypes.c_void_p(r)) if r else None))
    return results


class opmos_server:
    """Continuous-batching server (opmos_server_create/submit/poll/destroy)."""

    def __init__(self, graphs, options: Options | None = None, **kw):
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle.value for g in self.graphs])
        o = options or _options(**kw)
        h = ctypes.c_void_p()
        _check(lib().opmos_server_create(ctypes.cast(arr, ctypes.c_void_p), len(self.graphs), ctypes.byref(o),
                                         ctypes.byref(h)), "opmos_server_create")
        self.handle = h

    def submit(self, graph: int, d: int, start: int, goal: int) -> int:
        t = ctypes.c_uint64()
        _check(lib().opmos_server_submit(self.handle, graph, d, start, goal, ctypes.byref(t)), "opmos_server_submit")
        return int(t.value)

    def poll(self, ticket: int):
        """(PENDING, None) until done; then (status, Result or None)."""
        res = ctypes.c_void_p()
        rc = lib().opmos_server_poll(self.handle, ticket, ctypes.byref(res))
        if rc == PENDING:
            return PENDING, None
        if rc == OK:
            return OK, _take(res)
        if rc == ERR_INVALID_ARG and not res.value:
            _check(rc, "opmos_server_poll")
        return rc, None

    def close(self):
        if getattr(self, "handle", None):
            lib().opmos_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# test hooks (include/opmos_test.h): single device routines on given inputs
# ---------------------------------------------------------------------------
def opmos_test_merge(front, cand, cand_arc, block, slots: int = 32, lists: int = 1):
    """Device merge of one node (frontier rows ``front``, candidate rows
    ``cand`` with arc ids ``cand_arc``; the first ``slots`` in the node's
    slots, the rest in ``lists`` overflow lists) by one warp (block 0), one
    block (1) or a block merge split into ``block`` = 2..16 parts;
    returns (costs, origins) of the frontier after the merge (origin <
    len(front): that entry; else len(front) + candidate index)."""
    front = np.ascontiguousarray(front, np.uint32)
    cand = np.ascontiguousarray(cand, np.uint32)
    arc = np.ascontiguousarray(cand_arc, np.uint32)
    d = int(front.shape[1] if front.size else cand.shape[1])
    nf, nc = int(front.shape[0]), int(cand.shape[0])
    out = np.zeros((nf + nc + 1, d), np.uint32)
    org = np.zeros(nf + nc + 1, np.uint32)
    cnt = ctypes.c_uint32()
    _check(lib().opmos_test_merge(d, nf, _ptr(front), nc, _ptr(cand), _ptr(arc), int(block), slots, lists,
                                  _ptr(out), _ptr(org), ctypes.byref(cnt)), "opmos_test_merge")
    return out[:cnt.value], org[:cnt.value]


def opmos_test_window(f0, f1, dead, window: int, bins):
    """Device window selection and extraction over OPEN entries with
    F = (f0, f1); returns (taken bool array, b*)."""
    f0 = np.ascontiguousarray(f0, np.uint32)
    f1 = np.ascontiguousarray(f1, np.uint32)
    dead = np.ascontiguousarray(dead, np.uint8)
    bins = np.ascontiguousarray(bins, np.uint32)
    n = int(f0.shape[0])
    taken = np.zeros(max(n, 1), np.uint8)
    bstar = ctypes.c_uint32()
    _check(lib().opmos_test_window(n, _ptr(f0), _ptr(f1), _ptr(dead), window, _ptr(bins), _ptr(taken),
                                   ctypes.byref(bstar)), "opmos_test_window")
    return taken[:n].astype(bool), int(bstar.value)
