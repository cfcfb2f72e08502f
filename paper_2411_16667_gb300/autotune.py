"""Autotuner for the search launch parameters.

Chooses the window width W (labels extracted per step, the NUM_POP of
Sec. 5), the lanes per label of the expansion and the frontier tile size by
timing real solves through the C ABI on a calibration set: one query
(single-query mode) or a subset of a batch (batch mode). Every configuration
must return the same fronts as the first one -- a configuration that changes
a front is a bug, reported as an error. The choice is cached per (graph
digest, objectives used, mode) in memory and, optionally, in a JSON file.

The device work of each trial is the library's; this module only orders the
trials and keeps the fastest.
"""
from __future__ import annotations

import dataclasses
import hashlib
import itertools
import json
import os

import numpy as np

from . import opmos

# single queries: up to windows that take all of OPEN each step (on a
# latency-bound search, fewer and larger steps can win despite extra labels)
WINDOWS_SINGLE = (256, 1024, 4096, 16384, 65536, 262144)
WINDOWS_BATCH = (64, 256, 1024)
LANES = (4, 8, 16)
TILES = (32, 64)


@dataclasses.dataclass
class Choice:
    window: int
    lanes_per_label: int
    tile: int
    seconds: float
    table: list  # [(window, lanes, tile, seconds), ...]

    def options(self, **extra) -> opmos.Options:
        return opmos._options(window=self.window, lanes_per_label=self.lanes_per_label, tile=self.tile, **extra)


_cache: dict = {}


def graph_digest(graph: opmos.opmos_graph) -> str:
    h = hashlib.sha256()
    for a in (np.asarray([graph.n, graph.d], np.uint64), graph.rowptr, graph.col, graph.cost):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def _key(graph, d_used, mode):
    return f"{graph_digest(graph)}:d{d_used or graph.d}:{mode}"


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def autotune(graph: opmos.opmos_graph, queries, mode: str = "single", d_used: int = 0,
             windows=None, lanes=LANES, tiles=TILES, cache_path: str | None = None,
             stream_ptr: int | None = None) -> Choice:
    """Pick (W, lanes, tile). ``queries``: [(start, goal)] -- the first one in
    single mode, all of them (the calibration subset) in batch mode."""
    if mode not in ("single", "batch"):
        raise ValueError("mode must be 'single' or 'batch'")
    key = _key(graph, d_used, mode)
    if key in _cache:
        return _cache[key]
    disk = _load(cache_path)
    if key in disk:
        c = disk[key]
        ch = Choice(c["window"], c["lanes_per_label"], c["tile"], c["seconds"], c.get("table", []))
        _cache[key] = ch
        return ch
    windows = windows or (WINDOWS_SINGLE if mode == "single" else WINDOWS_BATCH)
    starts = [s for s, _ in queries]
    goals = [t for _, t in queries]
    heur = opmos.opmos_heur(graph, goals[0], d_used) if mode == "single" else None
    ref, table = None, []
    for w, l, t in itertools.product(windows, lanes, tiles):
        opt = opmos._options(window=w, lanes_per_label=l, tile=t, d_used=d_used or None,
                             flags=opmos.FLAG_NO_PATHS, stream=stream_ptr)
        if mode == "single":
            r = opmos.opmos_solve(graph, starts[0], goals[0], heur=heur, options=opt)
            fronts = [r.costs]
            secs = r.stats["search_ns"] / 1e9
        else:
            out = opmos.opmos_solve_batch(graph, starts, goals, options=opt)
            if any(st != opmos.OK for st, _ in out):
                continue
            fronts = [r.costs for _, r in out]
            secs = max(r.stats["search_ns"] for _, r in out) / 1e9
        if ref is None:
            ref = fronts
        elif any(not np.array_equal(a, b) for a, b in zip(ref, fronts)):
            raise RuntimeError(f"configuration W={w} lanes={l} tile={t} changed a front")
        table.append((w, l, t, secs))
    if not table:
        raise RuntimeError("no configuration completed the calibration set")
    best = min(table, key=lambda x: x[3])
    ch = Choice(best[0], best[1], best[2], best[3], table)
    _cache[key] = ch
    if cache_path:
        disk[key] = dataclasses.asdict(ch)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(disk, f, indent=1)
        os.replace(tmp, cache_path)
    return ch
