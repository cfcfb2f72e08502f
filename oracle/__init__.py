"""Sequential NAMOA* oracle (Algorithm 1) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never loads it. It shares no code with the CUDA path; the two
meet only in the arrays produced by ``synth``.

``namoa_oracle.cpp`` holds the algorithm; this file compiles it with the host
C++ compiler and wraps its C ABI with ctypes. Parity status: pinned (see the
header of ``namoa_oracle.cpp``).
"""
from __future__ import annotations

import contextlib
import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "namoa_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libnamoa_oracle.so")
_lock = threading.Lock()
_lib = None

STATS_FIELDS = ("extracted", "goal_extracted", "expanded", "candidates", "inserted",
                "pruned_open", "pruned_open_goal", "pruned_closed", "pruned_p",
                "comparisons", "max_open", "ns", "labels")

OK, INVALID, OVERFLOW, BUDGET, NOMEM = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle into ``libnamoa_oracle.so`` (plain g++, -O2)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    u32, u64, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    lib.oracle_heuristic.argtypes = [u32, u64, u32, p, p, p, u32, p]
    lib.oracle_solve.argtypes = [u32, u64, u32, p, p, p, p, u32, u32, u64, ctypes.POINTER(p)]
    lib.oracle_result_count.argtypes = [p]
    lib.oracle_result_count.restype = u32
    lib.oracle_result_costs.argtypes = [p, p]
    lib.oracle_result_path_len.argtypes = [p, u32]
    lib.oracle_result_path_len.restype = u32
    lib.oracle_result_path.argtypes = [p, u32, p, p]
    lib.oracle_result_stats.argtypes = [p, p]
    lib.oracle_result_free.argtypes = [p]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def library(path: str):
    """Run this binding on another build of ``namoa_oracle.cpp`` for the
    duration of the block: tests that plant a mistake in a copy of the
    oracle use it to show the pins catch the mistake."""
    global _lib
    saved = _lib
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _graph_arrays(g):
    return (np.ascontiguousarray(g.rowptr, np.uint64), np.ascontiguousarray(g.col, np.uint32),
            np.ascontiguousarray(g.cost, np.uint32))


def heuristic(g, goal: int) -> np.ndarray:
    """Ideal-point heuristic h[k, v] (uint32; 0xFFFFFFFF = goal unreachable)."""
    lib = _load()
    rp, col, cost = _graph_arrays(g)
    h = np.empty((g.d, g.n), np.uint32)
    rc = lib.oracle_heuristic(g.n, g.m, g.d, _ptr(rp), _ptr(col), _ptr(cost), goal, _ptr(h))
    if rc:
        raise OracleError(rc, "heuristic")
    return h


@dataclasses.dataclass
class Front:
    costs: np.ndarray  # uint32 [count, d], lexicographically sorted
    paths: list  # list of (nodes uint32 array, edges uint64 array)
    stats: dict


def solve(g, start: int, goal: int, h: np.ndarray | None = None, label_budget: int = 0,
          partial_ok: bool = False) -> Front:
    """Exact Pareto front of start->goal by Algorithm 1. With ``partial_ok``
    a run stopped by ``label_budget`` returns its counters (``stats['partial']
    = 1``) and an empty front instead of raising."""
    lib = _load()
    rp, col, cost = _graph_arrays(g)
    hp = None
    if h is not None:
        h = np.ascontiguousarray(h, np.uint32)
        hp = _ptr(h)
    res = ctypes.c_void_p()
    rc = lib.oracle_solve(g.n, g.m, g.d, _ptr(rp), _ptr(col), _ptr(cost), hp, start, goal,
                          label_budget, ctypes.byref(res))
    partial = rc == BUDGET and bool(res.value)
    if rc and not (partial and partial_ok):
        if res.value:
            lib.oracle_result_free(res)
        raise OracleError(rc, "solve")
    try:
        cnt = lib.oracle_result_count(res)
        costs = np.empty((cnt, g.d), np.uint32)
        if cnt:
            lib.oracle_result_costs(res, _ptr(costs))
        paths = []
        for i in range(cnt):
            ln = lib.oracle_result_path_len(res, i)
            nodes = np.empty(ln, np.uint32)
            edges = np.empty(max(ln - 1, 0), np.uint64)
            lib.oracle_result_path(res, i, _ptr(nodes), _ptr(edges) if edges.size else None)
            paths.append((nodes, edges))
        st = np.empty(len(STATS_FIELDS), np.uint64)
        lib.oracle_result_stats(res, _ptr(st))
        stats = {k: int(v) for k, v in zip(STATS_FIELDS, st)}
        stats["partial"] = int(partial)
    finally:
        lib.oracle_result_free(res)
    return Front(costs, paths, stats)
