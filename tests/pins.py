"""Independent reference facts the oracle is pinned to (pure Python, slow).

Nothing here imports the oracle or the CUDA library. Each helper restates a
textbook definition:

* ``brute_front``: the cost-unique non-dominated set of all simple s->t path
  costs, by depth-first enumeration (the definition in Sec. 3). With
  non-negative costs a non-simple path never adds a new non-dominated cost.
* ``dijkstra``: single-objective shortest distances (Dijkstra 1959).
* ``lex_dijkstra``: lexicographic-vector shortest distance; lexicographic
  order is a total order compatible with adding non-negative vectors, so
  Dijkstra's label-setting argument carries over.
* ``check_front``: mutual non-dominance, cost-uniqueness and path validity.
"""
from __future__ import annotations

import heapq

import numpy as np


def adjacency(g):
    """List of (v, arc_id) per node u."""
    rp = g.rowptr.astype(np.int64)
    return [[(int(g.col[e]), e) for e in range(rp[u], rp[u + 1])] for u in range(g.n)]


def dominates(a, b) -> bool:
    """a dominates b: a <= b in every objective and < in at least one (Sec. 3)."""
    return all(x <= y for x, y in zip(a, b)) and any(x < y for x, y in zip(a, b))


def nondominated_unique(vectors):
    """Cost-unique subset of vectors that no other vector dominates."""
    uniq = sorted(set(tuple(int(x) for x in v) for v in vectors))
    return [v for v in uniq if not any(dominates(w, v) for w in uniq)]


def brute_front(g, s: int, t: int, max_paths: int = 2_000_000):
    """Exact Pareto front (sorted list of tuples) by enumerating simple paths."""
    adj = adjacency(g)
    d = g.d
    cost = g.cost.astype(np.int64)
    found = []
    if s == t:
        return [tuple([0] * d)]
    on_path = [False] * g.n
    stack = [(s, iter(adj[s]), tuple([0] * d))]
    on_path[s] = True
    while stack:
        u, it, acc = stack[-1]
        nxt = next(it, None)
        if nxt is None:
            stack.pop()
            on_path[u] = False
            continue
        v, e = nxt
        if on_path[v]:
            continue
        acc2 = tuple(acc[k] + int(cost[k, e]) for k in range(d))
        if v == t:
            found.append(acc2)
            if len(found) > max_paths:
                raise RuntimeError("too many paths for brute force")
            continue
        on_path[v] = True
        stack.append((v, iter(adj[v]), acc2))
    return nondominated_unique(found)


def dijkstra(g, source: int, k: int = 0, reverse: bool = False):
    """Shortest distances under objective k from ``source`` (to ``source`` if
    ``reverse``); None where unreachable."""
    n = g.n
    rp = g.rowptr.astype(np.int64)
    nbr = [[] for _ in range(n)]
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            v = int(g.col[e])
            c = int(g.cost[k, e])
            if reverse:
                nbr[v].append((u, c))
            else:
                nbr[u].append((v, c))
    dist = [None] * n
    dist[source] = 0
    pq = [(0, source)]
    done = [False] * n
    while pq:
        du, u = heapq.heappop(pq)
        if done[u]:
            continue
        done[u] = True
        for v, c in nbr[u]:
            nd = du + c
            if dist[v] is None or nd < dist[v]:
                dist[v] = nd
                heapq.heappush(pq, (nd, v))
    return dist


def lex_dijkstra(g, s: int, t: int):
    """Lexicographically smallest s->t path cost vector (tuple) or None."""
    n, d = g.n, g.d
    rp = g.rowptr.astype(np.int64)
    cost = g.cost.astype(np.int64)
    best = [None] * n
    best[s] = tuple([0] * d)
    pq = [(best[s], s)]
    done = [False] * n
    while pq:
        du, u = heapq.heappop(pq)
        if done[u]:
            continue
        done[u] = True
        if u == t:
            return du
        for e in range(rp[u], rp[u + 1]):
            v = int(g.col[e])
            nd = tuple(du[k] + int(cost[k, e]) for k in range(d))
            if best[v] is None or nd < best[v]:
                best[v] = nd
                heapq.heappush(pq, (nd, v))
    return None


def check_front(g, s: int, t: int, costs: np.ndarray, paths) -> None:
    """Assert the Sec. 3 output contract: cost-unique, mutually non-dominated,
    and each path is an s->t walk along existing arcs whose cost sum equals
    its reported vector."""
    vecs = [tuple(int(x) for x in row) for row in costs]
    assert len(set(vecs)) == len(vecs), "front is not cost-unique"
    for a in vecs:
        for b in vecs:
            assert not dominates(a, b), f"{a} dominates {b}"
    assert len(paths) == len(vecs)
    rp = g.rowptr.astype(np.int64)
    for vec, (nodes, edges) in zip(vecs, paths):
        nodes = [int(x) for x in nodes]
        edges = [int(x) for x in edges]
        assert nodes[0] == s and nodes[-1] == t
        assert len(edges) == len(nodes) - 1
        acc = [0] * g.d
        for i, e in enumerate(edges):
            u, v = nodes[i], nodes[i + 1]
            assert rp[u] <= e < rp[u + 1], f"arc {e} does not leave node {u}"
            assert int(g.col[e]) == v, f"arc {e} does not enter node {v}"
            for k in range(g.d):
                acc[k] += int(g.cost[k, e])
        assert tuple(acc) == vec, f"path sum {acc} != label {vec}"


def load_front_fixture(path: str):
    """Parse a tests/golden/*.front file: returns (meta dict, costs array)."""
    meta = {}
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, _, rest = line.partition(" ")
            if head == "graph":
                meta["name"], meta["digest"] = rest.split()
            elif head == "query":
                meta["start"], meta["goal"] = (int(x) for x in rest.split())
            elif head == "d":
                meta["d"] = int(rest)
            elif head == "stats":
                meta["stats"] = {k: int(v) for k, v in (kv.split("=") for kv in rest.split())}
            elif head == "count":
                meta["count"] = int(rest)
            else:
                rows.append([int(x) for x in line.split()])
    costs = np.array(rows, dtype=np.uint32).reshape(-1, meta.get("d", 1))
    return meta, costs


def check_front_sampled(g, s: int, t: int, costs: np.ndarray, paths, nrows: int = 1000, npaths: int = 100,
                        seed: int = 0) -> None:
    """The check_front contract for large fronts: cost-uniqueness on every
    row, non-dominance for a sample of rows against every row (vectorised),
    and path validity for a sample of paths."""
    c = np.asarray(costs, dtype=np.int64)
    assert np.unique(c, axis=0).shape[0] == c.shape[0], "front is not cost-unique"
    rng = np.random.default_rng(seed)
    rows = rng.choice(c.shape[0], size=min(nrows, c.shape[0]), replace=False)
    for r in rows:
        le = np.all(c <= c[r], axis=1) & np.any(c < c[r], axis=1)
        assert not le.any(), f"row {r} is dominated"
    sel = rng.choice(len(paths), size=min(npaths, len(paths)), replace=False)
    check_front(g, s, t, c[sel], [paths[i] for i in sel])
