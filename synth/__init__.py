"""Seeded synthetic multi-objective graphs and start/goal queries.

This module builds inputs only. It holds none of the search method's
arithmetic (no dominance test, no heuristic, no path-cost sum): the oracle
under ``oracle/`` and the CUDA library both take what it produces as plain
arrays. Everything is driven by one counter-based generator (SplitMix64's
output function over ``seed``/``stream``/``index``), so a workload is a pure
function of its seed on every platform.

Graph format (the same one the C ABI takes, see the problem statement of
Sec. 3): ``n`` nodes, ``m`` directed arcs in CSR order (``rowptr`` uint64 of
length n+1, ``col`` uint32 of length m), ``d`` objectives with non-negative
uint32 costs stored structure-of-arrays, ``cost[k*m + e]``.

Workloads (shapes of the paper's ship-routing graphs, Sec. 6.1 / Table 2,
scaled up; the TMPLAR/ERA5 graphs themselves are not available):

* ``config1``  32x32 8-connected grid, d=2, arc costs U[1,10] i.i.d.
* ``config2``  256x256 8-connected ship grid, d=3: move length (10/14),
  length x current factor, length x wave factor; factors in [1,8] from
  smooth 32-blob fields; 5% land.
* ``config3``  200k uniform points, symmetric 4-NN road-like graph, d=4;
  256 queries with hop distance U[50,400].
* ``config4``  the config-2 grid plus an exposure field and a step count,
  d=5; 1,024 queries with Chebyshev distance U[16,128].
* ``time_route`` a time-expanded ship route (cells x time windows, two
  speeds per move) with up to 12 objectives in the order of Table 1, for the
  high objective counts of the paper's routes (Sec. 6.1, Tables 1-2).
* ``random_digraph`` / ``small_grid``: tiny graphs with ties and zero costs.
"""
from __future__ import annotations

import dataclasses
import functools
import hashlib

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014), wrapping uint64."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def rand_u64(seed: int, stream: int, index) -> np.ndarray:
    """Counter-based uint64 draw number ``index`` of ``stream`` under ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) * _STREAM_MUL))
        return _mix64(key + (idx + np.uint64(1)) * _GAMMA)


def rand_int(seed: int, stream: int, index, lo: int, hi: int) -> np.ndarray:
    """Uniform integers in [lo, hi] (inclusive) by 32x32 multiply-high."""
    span = np.uint64(hi - lo + 1)
    u = rand_u64(seed, stream, index) >> np.uint64(32)
    return (np.uint64(lo) + ((u * span) >> np.uint64(32))).astype(np.int64)


def rand_unit(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    u = rand_u64(seed, stream, index) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Graph:
    """A directed multi-objective graph in CSR form with SoA uint32 costs."""

    name: str
    n: int
    d: int
    rowptr: np.ndarray  # uint64 [n+1]
    col: np.ndarray  # uint32 [m]
    cost: np.ndarray  # uint32 [d, m], C-contiguous
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def first_objectives(self, d: int) -> "Graph":
        """The same graph restricted to its first ``d`` objectives (Table 1 order rule)."""
        assert 1 <= d <= self.d
        return Graph(f"{self.name}[:{d}]", self.n, d, self.rowptr, self.col,
                     np.ascontiguousarray(self.cost[:d]), dict(self.meta))

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (np.asarray([self.n, self.d], np.uint64), self.rowptr, self.col, self.cost):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()[:16]

    def src(self) -> np.ndarray:
        """Source node of every arc (uint32 [m])."""
        deg = np.diff(self.rowptr).astype(np.int64)
        return np.repeat(np.arange(self.n, dtype=np.uint32), deg)


def _csr_from_arcs(n: int, src: np.ndarray, dst: np.ndarray, cost: np.ndarray):
    """Sort arcs by (src, dst) and build CSR; cost is [d, m] in the input arc order."""
    order = np.lexsort((dst, src))
    src, dst, cost = src[order], dst[order], cost[:, order]
    rowptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(src, minlength=n), out=rowptr[1:])
    return rowptr, dst.astype(np.uint32), np.ascontiguousarray(cost.astype(np.uint32))


# --------------------------------------------------------------------------
# 8-connected grids
# --------------------------------------------------------------------------
_NBR8 = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def grid8_arcs(rows: int, cols: int, open_mask: np.ndarray | None = None):
    """Directed arcs of an 8-connected grid in CSR order (by source, then the
    fixed neighbour order of ``_NBR8``). Node id = r*cols + c. An arc exists
    when both cells are open; diagonal moves may cut corners.

    Returns (src, dst, is_diagonal) as int64/int64/bool arrays."""
    r = np.arange(rows)[:, None]
    c = np.arange(cols)[None, :]
    srcs, dsts, diags = [], [], []
    for dr, dc in _NBR8:
        rr, cc = r + dr, c + dc
        ok = (rr >= 0) & (rr < rows) & (cc >= 0) & (cc < cols)
        ok = np.broadcast_to(ok, (rows, cols))
        uu = np.broadcast_to(r * cols + c, (rows, cols))[ok]
        vv = np.broadcast_to(rr * cols + cc, (rows, cols))[ok]
        srcs.append(uu)
        dsts.append(vv)
        diags.append(np.full(uu.shape, dr != 0 and dc != 0))
    src = np.concatenate(srcs).astype(np.int64)
    dst = np.concatenate(dsts).astype(np.int64)
    diag = np.concatenate(diags)
    if open_mask is not None:
        flat = open_mask.reshape(-1)
        keep = flat[src] & flat[dst]
        src, dst, diag = src[keep], dst[keep], diag[keep]
    # CSR order: by source, then neighbour order (stable sort keeps _NBR8 order)
    order = np.argsort(src, kind="stable")
    return src[order], dst[order], diag[order]


def _rowptr(n: int, src: np.ndarray) -> np.ndarray:
    rowptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(src, minlength=n), out=rowptr[1:])
    return rowptr


def config1(seed: int = 1) -> tuple[Graph, list[tuple[int, int]]]:
    """32x32 8-connected grid, d=2, per-arc costs U[1,10] drawn in CSR order."""
    rows = cols = 32
    n = rows * cols
    src, dst, _ = grid8_arcs(rows, cols)
    m = src.shape[0]
    cost = np.empty((2, m), np.uint32)
    for k in range(2):
        cost[k] = rand_int(seed, 100 + k, np.arange(m), 1, 10)
    g = Graph("grid32-d2", n, 2, _rowptr(n, src), dst.astype(np.uint32), cost,
              {"rows": rows, "cols": cols, "seed": seed})
    return g, [(0, n - 1)]


def blob_field(seed: int, stream: int, rows: int, cols: int, nblobs: int = 32) -> np.ndarray:
    """Smooth field: sum of ``nblobs`` isotropic Gaussian blobs with centres
    uniform over the grid, sigma U[8,48] cells, amplitude U[0.5,1]; min-max
    normalised to [0,1]. Evaluated in float64 on the host."""
    i = np.arange(nblobs)
    cy = rand_unit(seed, stream, 4 * i) * rows
    cx = rand_unit(seed, stream, 4 * i + 1) * cols
    sig = 8.0 + 40.0 * rand_unit(seed, stream, 4 * i + 2)
    amp = 0.5 + 0.5 * rand_unit(seed, stream, 4 * i + 3)
    y = np.arange(rows, dtype=np.float64)[:, None]
    x = np.arange(cols, dtype=np.float64)[None, :]
    f = np.zeros((rows, cols))
    for b in range(nblobs):
        f += amp[b] * np.exp(-((y - cy[b]) ** 2 + (x - cx[b]) ** 2) / (2.0 * sig[b] ** 2))
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)


def _edge_factor(field: np.ndarray, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Integer factor in [1,8] from the field at the arc midpoint (mean of the
    two endpoint cells), round half up. Symmetric in (src, dst)."""
    flat = field.reshape(-1)
    fm = 0.5 * (flat[src] + flat[dst])
    return np.clip(np.floor(1.0 + 7.0 * fm + 0.5), 1, 8).astype(np.int64)


def _components(n: int, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    a = sp.csr_matrix((np.ones(src.shape[0], np.int8), (src, dst)), shape=(n, n))
    return csg.connected_components(a, directed=True, connection="weak")[1]


@functools.lru_cache(maxsize=4)
def _ship_grid(seed: int, rows: int = 256, cols: int = 256):
    """Fields and land mask shared by configs 2 and 4."""
    n = rows * cols
    current = blob_field(seed, 200, rows, cols)
    wave = blob_field(seed, 201, rows, cols)
    exposure = blob_field(seed, 202, rows, cols)
    s, t = 0, n - 1
    for sub in range(64):
        landf = blob_field(seed, 300 + sub, rows, cols).reshape(-1)
        nland = int(0.05 * n)
        order = np.lexsort((np.arange(n), -landf))  # highest first, ties by index
        open_mask = np.ones(n, bool)
        open_mask[order[:nland]] = False
        open_mask[s] = open_mask[t] = True
        src, dst, diag = grid8_arcs(rows, cols, open_mask.reshape(rows, cols))
        comp = _components(n, src, dst)
        if comp[s] == comp[t]:
            return dict(rows=rows, cols=cols, current=current, wave=wave, exposure=exposure,
                        open=open_mask, src=src, dst=dst, diag=diag, comp=comp, land_sub=sub)
    raise RuntimeError("no land mask connects start and goal")


def config2(seed: int = 1) -> tuple[Graph, list[tuple[int, int]]]:
    """256x256 ship grid, d=3: length, length x current, length x wave."""
    sg = _ship_grid(seed)
    n = sg["rows"] * sg["cols"]
    src, dst = sg["src"], sg["dst"]
    length = np.where(sg["diag"], 14, 10).astype(np.int64)
    cost = np.stack([length,
                     length * _edge_factor(sg["current"], src, dst),
                     length * _edge_factor(sg["wave"], src, dst)]).astype(np.uint32)
    g = Graph("ship256-d3", n, 3, _rowptr(n, src), dst.astype(np.uint32), np.ascontiguousarray(cost),
              {"rows": sg["rows"], "cols": sg["cols"], "seed": seed, "land_sub": sg["land_sub"]})
    return g, [(0, n - 1)]


def ship_grid(seed: int, rows: int, d: int = 3) -> tuple[Graph, list[tuple[int, int]]]:
    """A rows x rows version of the config-2 ship grid (same field recipe,
    5% land, corner to corner), for test sizes; d <= 5 uses the config-4
    objective list (length, time, fuel, exposure, steps)."""
    sg = _ship_grid(seed, rows, rows)
    n = rows * rows
    src, dst = sg["src"], sg["dst"]
    length = np.where(sg["diag"], 14, 10).astype(np.int64)
    objs = [length, length * _edge_factor(sg["current"], src, dst), length * _edge_factor(sg["wave"], src, dst),
            _edge_factor(sg["exposure"], src, dst), np.ones_like(length)]
    cost = np.stack(objs[:d]).astype(np.uint32)
    g = Graph(f"ship{rows}-d{d}-s{seed}", n, d, _rowptr(n, src), dst.astype(np.uint32), np.ascontiguousarray(cost),
              {"rows": rows, "cols": rows, "seed": seed, "land_sub": sg["land_sub"]})
    return g, [(0, n - 1)]


def config4(seed: int = 1, nq: int = 1024) -> tuple[Graph, list[tuple[int, int]]]:
    """Config-2 grid plus obj4 = exposure factor in [1,8] and obj5 = 1 per move;
    ``nq`` queries with Chebyshev distance U[16,128] between reachable open cells."""
    sg = _ship_grid(seed)
    rows, cols = sg["rows"], sg["cols"]
    n = rows * cols
    src, dst = sg["src"], sg["dst"]
    length = np.where(sg["diag"], 14, 10).astype(np.int64)
    cost = np.stack([length,
                     length * _edge_factor(sg["current"], src, dst),
                     length * _edge_factor(sg["wave"], src, dst),
                     _edge_factor(sg["exposure"], src, dst),
                     np.ones_like(length)]).astype(np.uint32)
    g = Graph("ship256-d5", n, 5, _rowptr(n, src), dst.astype(np.uint32), np.ascontiguousarray(cost),
              {"rows": rows, "cols": cols, "seed": seed, "land_sub": sg["land_sub"]})
    open_cells = np.flatnonzero(sg["open"])
    comp = sg["comp"]
    rr, cc = np.divmod(np.arange(n), cols)
    queries = []
    ctr = 0
    while len(queries) < nq:
        s = int(open_cells[rand_int(seed, 400, ctr, 0, open_cells.size - 1)])
        r = int(rand_int(seed, 401, ctr, 16, 128))
        ctr += 1
        cheb = np.maximum(np.abs(rr - rr[s]), np.abs(cc - cc[s]))
        cand = np.flatnonzero((cheb == r) & sg["open"] & (comp == comp[s]))
        if cand.size == 0:
            continue
        t = int(cand[rand_int(seed, 402, ctr, 0, cand.size - 1)])
        queries.append((s, t))
    return g, queries


# --------------------------------------------------------------------------
# Road-like 4-NN graph
# --------------------------------------------------------------------------
def _bfs_hops(adj, s: int, max_hops: int) -> np.ndarray:
    """Hop distance from ``s`` (-1 beyond ``max_hops`` or unreachable)."""
    import scipy.sparse.csgraph as csg
    dist = csg.dijkstra(adj, directed=True, indices=s, unweighted=True, limit=max_hops + 0.5)
    return np.where(np.isfinite(dist), dist, -1).astype(np.int64)


@functools.lru_cache(maxsize=2)
def config3(seed: int = 1, nq: int = 256, npts: int = 200_000) -> tuple[Graph, list[tuple[int, int]]]:
    """Uniform points in the unit square (20-bit integer coordinates), edge
    {u,v} iff v is among u's 4 nearest neighbours or u among v's (distance
    ties by index). Per undirected edge: obj1 = round(1e4 * length),
    obj2 = obj1 * U{1..4}, obj3 = U[0,50], obj4 = U[1,100]. Queries: random s,
    hop target U[50,400], t uniform among nodes at that hop distance."""
    from scipy.spatial import cKDTree
    scale = 1 << 20
    ix = rand_int(seed, 500, np.arange(npts), 0, scale - 1)
    iy = rand_int(seed, 501, np.arange(npts), 0, scale - 1)
    pts = np.stack([ix, iy], 1).astype(np.float64)  # exact integers in float64
    tree = cKDTree(pts)
    kq = 9
    _, nbr = tree.query(pts, k=kq)
    nbr = nbr.astype(np.int64)
    dx = ix[nbr] - ix[:, None]
    dy = iy[nbr] - iy[:, None]
    d2 = dx * dx + dy * dy  # exact in int64
    selfm = nbr == np.arange(npts)[:, None]
    d2 = np.where(selfm, np.iinfo(np.int64).max, d2)
    order = np.lexsort((nbr, d2), axis=1)[:, :4]
    knn = np.take_along_axis(nbr, order, 1)
    u = np.repeat(np.arange(npts), 4)
    v = knn.reshape(-1)
    a, b = np.minimum(u, v), np.maximum(u, v)
    pairs = np.unique(a * npts + b)
    a, b = pairs // npts, pairs % npts
    ne = a.shape[0]
    ddx, ddy = ix[a] - ix[b], iy[a] - iy[b]
    length = np.sqrt((ddx * ddx + ddy * ddy).astype(np.float64)) / scale
    o1 = np.floor(1e4 * length + 0.5).astype(np.int64)
    eidx = np.arange(ne)
    o2 = o1 * rand_int(seed, 510, eidx, 1, 4)
    o3 = rand_int(seed, 511, eidx, 0, 50)
    o4 = rand_int(seed, 512, eidx, 1, 100)
    cu = np.stack([o1, o2, o3, o4])
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    cost = np.concatenate([cu, cu], 1)
    rowptr, col, cost = _csr_from_arcs(npts, src, dst, cost)
    g = Graph("knn200k-d4", npts, 4, rowptr, col, cost, {"seed": seed, "undirected_edges": int(ne)})
    import scipy.sparse as sp
    adj = sp.csr_matrix((np.ones(col.shape[0], np.float64), col.astype(np.int64), rowptr.astype(np.int64)),
                        shape=(npts, npts))
    queries = []
    ctr = 0
    while len(queries) < nq:
        s = int(rand_int(seed, 520, ctr, 0, npts - 1))
        h = int(rand_int(seed, 521, ctr, 50, 400))
        ctr += 1
        hop = _bfs_hops(adj, s, h)
        cand = np.flatnonzero(hop == h)
        if cand.size == 0:
            continue
        t = int(cand[rand_int(seed, 522, ctr, 0, cand.size - 1)])
        queries.append((s, t))
    return g, queries


# --------------------------------------------------------------------------
# Time-expanded ship routes (high objective counts)
# --------------------------------------------------------------------------
ROUTE_OBJECTIVES = ("distance", "fuel", "roll", "pitch", "vertical acceleration", "horizontal acceleration",
                    "vertical bending moment", "vertical shear force", "wave height", "wave period",
                    "relative wave bearing", "random")


def _drifting_field(seed: int, stream: int, rows: int, cols: int, windows: int, nblobs: int = 6) -> np.ndarray:
    """A smooth field per time window: ``nblobs`` Gaussian blobs (sigma
    U[1.5, 4] cells, amplitude U[0.5, 1]) whose centres drift by a fixed
    seeded velocity (up to 0.6 cells per window); min-max normalised to [0, 1]
    over all windows. Shape [windows, rows, cols]."""
    i = np.arange(nblobs)
    cy = rand_unit(seed, stream, 6 * i) * rows
    cx = rand_unit(seed, stream, 6 * i + 1) * cols
    vy = (rand_unit(seed, stream, 6 * i + 2) - 0.5) * 1.2
    vx = (rand_unit(seed, stream, 6 * i + 3) - 0.5) * 1.2
    sig = 1.5 + 2.5 * rand_unit(seed, stream, 6 * i + 4)
    amp = 0.5 + 0.5 * rand_unit(seed, stream, 6 * i + 5)
    y = np.arange(rows, dtype=np.float64)[None, :, None]
    x = np.arange(cols, dtype=np.float64)[None, None, :]
    w = np.arange(windows, dtype=np.float64)[:, None, None]
    f = np.zeros((windows, rows, cols))
    for b in range(nblobs):
        f += amp[b] * np.exp(-((y - cy[b] - vy[b] * w) ** 2 + (x - cx[b] - vx[b] * w) ** 2) / (2.0 * sig[b] ** 2))
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)


def time_route(seed: int, rows: int, cols: int, windows: int = 10, d: int = 12) -> tuple[Graph, list[tuple[int, int]]]:
    """A time-expanded ship route shaped like the paper's TMPLAR graphs
    (Sec. 6.1: a reduced corridor, each location expanded into time windows,
    up to 12 objectives used in the order of Table 1), from seeded drifting
    weather fields instead of ERA5 data.

    Nodes: (cell, window) for the rows x cols 8-connected cells and
    ``windows`` time windows, id = cell * windows + window, plus one goal node
    (id rows*cols*windows) that every window of the destination cell reaches
    at zero cost. A move to a neighbouring cell departs in window w and
    arrives in window w+1 (fast, speed 3), w+2 (speed 2) or w+3 (slow, speed
    1); moves past the last window do not exist. Start: cell (0, 0) in window 0; destination: cell
    (rows-1, cols-1).

    Objectives of a move (integers, all >= 0), from seven wave-height
    components h0..h6, the wave period p and the wave direction (fields at
    the move's midpoint in its departure window, each in [0, 1]), the
    relative bearing b in [0, 1] (0 following seas, 1 head seas), the move
    length L (10 straight, 14 diagonal) and the speed s (1, 2 or 3):
      distance L; fuel round(L (s + 2h0)); roll round(L (1 + 8h1 sin(pi b)));
      pitch round(L (1 + 8h2 b)); vertical acceleration round(L (1 + 4h3 b s^2));
      horizontal acceleration round(L (1 + 4h4 sin(pi b) s)); vertical
      bending moment round(L (1 + 6h5 p)); vertical shear force
      round(L (1 + 6h6 (1 - p))); wave height round(L/10 (10 + 70h0)); wave
      period round(L/10 (10 + 70p)); relative wave bearing round(8Lb);
      random U[1, 100] per arc."""
    assert 1 <= d <= len(ROUTE_OBJECTIVES) and rows >= 1 and cols >= 1 and windows >= 2
    # seven wave-height components (one per response objective), the period
    # and the direction
    HS = [_drifting_field(seed, 1220 + j, rows, cols, windows) for j in range(7)]
    Pd = _drifting_field(seed, 1201, rows, cols, windows)
    TH = _drifting_field(seed, 1202, rows, cols, windows) * (2.0 * np.pi)
    csrc, cdst, diag = grid8_arcs(rows, cols)
    ncell = rows * cols
    goal = ncell * windows
    n = goal + 1
    srcs, dsts, objs = [], [], []
    length = np.where(diag, 14, 10).astype(np.float64)
    r0, c0 = csrc // cols, csrc % cols
    r1, c1 = cdst // cols, cdst % cols
    bearing = np.arctan2(r1 - r0, c1 - c0)
    for speed, tau in ((3, 1), (2, 2), (1, 3)):
        for w in range(windows - tau):
            hs = [0.5 * (f[w].reshape(-1)[csrc] + f[w].reshape(-1)[cdst]) for f in HS]
            pf, tf = Pd[w].reshape(-1), TH[w].reshape(-1)
            p = 0.5 * (pf[csrc] + pf[cdst])
            th = 0.5 * (tf[csrc] + tf[cdst])
            rel = np.abs(np.angle(np.exp(1j * (bearing - th)))) / np.pi  # 0 following, 1 head seas
            L10 = length / 10.0
            sb = np.sin(np.pi * rel)
            idx = np.arange(csrc.shape[0]) + csrc.shape[0] * (w + windows * (speed - 1))
            o = [length,
                 length * (speed + 2.0 * hs[0]),
                 length * (1.0 + 8.0 * hs[1] * sb),
                 length * (1.0 + 8.0 * hs[2] * rel),
                 length * (1.0 + 4.0 * hs[3] * rel * speed * speed),
                 length * (1.0 + 4.0 * hs[4] * sb * speed),
                 length * (1.0 + 6.0 * hs[5] * p),
                 length * (1.0 + 6.0 * hs[6] * (1.0 - p)),
                 L10 * (10.0 + 70.0 * hs[0]),
                 L10 * (10.0 + 70.0 * p),
                 L10 * 80.0 * rel,
                 rand_int(seed, 1210, idx, 1, 100).astype(np.float64)]
            srcs.append(csrc * windows + w)
            dsts.append(cdst * windows + w + tau)
            objs.append(np.floor(np.stack(o[:d]) + 0.5).astype(np.int64))
    dest = ncell - 1
    sink_src = dest * windows + np.arange(windows)
    srcs.append(sink_src)
    dsts.append(np.full(windows, goal))
    objs.append(np.zeros((d, windows), np.int64))
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    cost = np.concatenate(objs, axis=1)
    rowptr, col, cost = _csr_from_arcs(n, src, dst, cost)
    g = Graph(f"route{rows}x{cols}x{windows}-d{d}-s{seed}", n, d, rowptr, col, cost,
              {"rows": rows, "cols": cols, "windows": windows, "seed": seed,
               "objectives": ROUTE_OBJECTIVES[:d]})
    return g, [(0, goal)]


# --------------------------------------------------------------------------
# Tiny graphs for pins and edge cases
# --------------------------------------------------------------------------
def random_digraph(seed: int, n: int, d: int, p: float = 0.3, cmax: int = 3,
                   cmin: int = 0) -> Graph:
    """Random digraph: arc (u,v), u != v, with probability ``p``; costs
    U[cmin, cmax] per objective (small ranges force ties and zero arcs)."""
    uu, vv = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    uu, vv = uu.reshape(-1), vv.reshape(-1)
    keep = (uu != vv) & (rand_unit(seed, 600, np.arange(n * n)) < p)
    src, dst = uu[keep], vv[keep]
    m = src.shape[0]
    cost = np.stack([rand_int(seed, 610 + k, np.arange(m), cmin, cmax) for k in range(d)]) \
        if m else np.zeros((d, 0), np.int64)
    rowptr, col, cost = _csr_from_arcs(n, src, dst, cost.reshape(d, m))
    return Graph(f"rand{n}-d{d}-s{seed}", n, d, rowptr, col, cost, {"seed": seed})


def small_grid(seed: int, rows: int, cols: int, d: int, cmin: int = 1, cmax: int = 10) -> Graph:
    """rows x cols 8-connected grid with per-arc costs U[cmin,cmax]."""
    src, dst, _ = grid8_arcs(rows, cols)
    n, m = rows * cols, src.shape[0]
    cost = np.stack([rand_int(seed, 700 + k, np.arange(m), cmin, cmax) for k in range(d)])
    return Graph(f"grid{rows}x{cols}-d{d}-s{seed}", n, d, _rowptr(n, src), dst.astype(np.uint32),
                 np.ascontiguousarray(cost.astype(np.uint32)), {"rows": rows, "cols": cols})


def from_arcs(n: int, arcs: list[tuple[int, int, tuple[int, ...]]], name: str = "custom") -> Graph:
    """Graph from an explicit arc list [(u, v, (c_0, ..., c_{d-1})), ...]."""
    d = len(arcs[0][2]) if arcs else 1
    src = np.array([a[0] for a in arcs], np.int64)
    dst = np.array([a[1] for a in arcs], np.int64)
    cost = np.array([a[2] for a in arcs], np.int64).T.reshape(d, len(arcs))
    rowptr, col, cost = _csr_from_arcs(n, src, dst, cost)
    return Graph(name, n, d, rowptr, col, cost, {})


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}
