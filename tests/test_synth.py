"""The seeded input generators against the recipes they state (CPU only).

The generators carry none of the method's arithmetic; these checks make sure
the workloads are the graphs the benchmark configs describe: sizes, move
sets, cost ranges and their relations, symmetry, land, and query distances.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import synth


def _arcs(g):
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr.astype(np.int64)))
    return src, g.col.astype(np.int64)


def _reverse_index(g):
    """For every arc u->v, the index of the arc v->u (asserts it exists)."""
    src, dst = _arcs(g)
    key = src * g.n + dst
    order = np.argsort(key, kind="stable")
    rkey = dst * g.n + src
    pos = np.searchsorted(key[order], rkey)
    assert np.all(pos < key.size) and np.array_equal(key[order][np.minimum(pos, key.size - 1)], rkey), \
        "some arc has no reverse arc"
    return order[pos]


def _hops(g, s, t):
    a = sp.csr_matrix((np.ones(g.m), g.col.astype(np.int64), g.rowptr.astype(np.int64)), shape=(g.n, g.n))
    return int(shortest_path(a, unweighted=True, indices=[s])[0, t])


def test_splitmix64_output_function_matches_published_sequence():
    """SplitMix64 seeded with 0 (Steele, Lea, Flood 2014): state advances by
    the golden gamma, and the first two outputs are the published values."""
    gamma = 0x9E3779B97F4A7C15
    assert int(synth._mix64(np.uint64(gamma))) == 0xE220A8397B1DCDAF
    assert int(synth._mix64(np.uint64((2 * gamma) % 2**64))) == 0x6E789E6AA1B965F4


def test_counter_based_draws_are_deterministic_and_in_range():
    a = synth.rand_int(7, 3, np.arange(10000), 1, 10)
    assert np.array_equal(a, synth.rand_int(7, 3, np.arange(10000), 1, 10))
    assert a.min() == 1 and a.max() == 10
    assert not np.array_equal(a, synth.rand_int(7, 4, np.arange(10000), 1, 10))
    u = synth.rand_unit(7, 3, np.arange(10000))
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.02


def test_config1_recipe():
    g, q = synth.config1()
    assert (g.n, g.d, g.m) == (1024, 2, 7812)
    assert g.cost.min() >= 1 and g.cost.max() <= 10
    assert q == [(0, 1023)]
    src, dst = _arcs(g)
    r0, c0 = np.divmod(src, 32)
    r1, c1 = np.divmod(dst, 32)
    assert np.all(np.maximum(np.abs(r0 - r1), np.abs(c0 - c1)) == 1), "not an 8-connected move"


def test_config2_recipe():
    g, q = synth.config2()
    assert (g.n, g.d) == (65536, 3) and q == [(0, 65535)]
    src, dst = _arcs(g)
    r0, c0 = np.divmod(src, 256)
    r1, c1 = np.divmod(dst, 256)
    assert np.all(np.maximum(np.abs(r0 - r1), np.abs(c0 - c1)) == 1)
    diag = (r0 != r1) & (c0 != c1)
    assert np.array_equal(g.cost[0], np.where(diag, 14, 10)), "length is 10 straight, 14 diagonal"
    for k in (1, 2):
        f = g.cost[k] // g.cost[0]
        assert np.array_equal(f * g.cost[0], g.cost[k]) and f.min() >= 1 and f.max() <= 8
        assert len(np.unique(f)) >= 6, "factor field is not spread over [1,8]"
    rev = _reverse_index(g)
    assert np.array_equal(g.cost[:, rev], g.cost), "costs are not symmetric"
    deg = np.diff(g.rowptr.astype(np.int64))
    land = int(0.05 * g.n)
    assert land <= int((deg == 0).sum()) <= land + 64, "about 5% of the cells are land"
    assert deg[0] > 0 and deg[g.n - 1] > 0


def test_config4_recipe():
    g, q = synth.config4(1, nq=48)
    g2, _ = synth.config2()
    assert (g.n, g.d) == (65536, 5) and len(q) == 48
    assert np.array_equal(g.cost[:3], g2.cost) and np.array_equal(g.rowptr, g2.rowptr)
    assert g.cost[3].min() >= 1 and g.cost[3].max() <= 8, "exposure factor in [1,8]"
    assert np.all(g.cost[4] == 1), "one step per move"
    deg = np.diff(g.rowptr.astype(np.int64))
    for s, t in q[:16]:
        (rs, cs), (rt, ct) = divmod(s, 256), divmod(t, 256)
        assert 16 <= max(abs(rs - rt), abs(cs - ct)) <= 128
        assert deg[s] > 0 and deg[t] > 0
        assert np.isfinite(_hops(g, s, t)), "goal not reachable"


@pytest.fixture(scope="module")
def road():
    return synth.config3()


def test_config3_recipe(road):
    g, q = road
    assert (g.n, g.d) == (200000, 4) and len(q) == 256
    rev = _reverse_index(g)
    assert np.array_equal(g.cost[:, rev], g.cost), "per-undirected-edge costs"
    deg = np.diff(g.rowptr.astype(np.int64))
    assert deg.min() >= 4, "every node keeps its 4 nearest neighbours"
    o1, o2, o3, o4 = (c.astype(np.int64) for c in g.cost)
    pos = o1 > 0
    assert np.all(o2[~pos] == 0)
    mult = o2[pos] // o1[pos]
    assert np.array_equal(mult * o1[pos], o2[pos]) and mult.min() == 1 and mult.max() == 4
    assert o3.min() >= 0 and o3.max() <= 50
    assert o4.min() >= 1 and o4.max() <= 100
    # lengths: 1e4 x the Euclidean length in the unit square, ~N^-1/2 apart
    assert 10 < np.median(o1) < 100


def test_config3_query_hops(road):
    g, q = road
    for s, t in q[:8]:
        assert 50 <= _hops(g, s, t) <= 400


def test_time_route_recipe():
    """Time-expanded route: (cell, window) nodes plus a goal node; a move
    arrives 1, 2 or 3 windows after it departs (speeds 3, 2, 1); the goal is
    entered from every window of the destination cell at zero cost; the first
    objectives keep the order of Table 1 and the stated ranges."""
    rows, cols, w, d = 3, 4, 8, 12
    g, q = synth.time_route(1, rows, cols, w, d)
    ncell = rows * cols
    goal = ncell * w
    assert (g.n, g.d) == (goal + 1, 12) and q == [(0, goal)]
    assert g.meta["objectives"][:2] == ("distance", "fuel") and g.meta["objectives"][-1] == "random"
    src, dst = _arcs(g)
    into_goal = dst == goal
    assert np.array_equal(np.sort(src[into_goal]), (ncell - 1) * w + np.arange(w))
    assert np.all(g.cost[:, into_goal] == 0)
    assert np.diff(g.rowptr.astype(np.int64))[goal] == 0, "the goal has no out-arcs"
    mv = ~into_goal
    cu, wu = np.divmod(src[mv], w)
    cv, wv = np.divmod(dst[mv], w)
    tau = wv - wu
    assert set(np.unique(tau)) == {1, 2, 3}
    ru, cu_ = np.divmod(cu, cols)
    rv, cv_ = np.divmod(cv, cols)
    cheb = np.maximum(np.abs(ru - rv), np.abs(cu_ - cv_))
    assert np.all(cheb == 1), "moves go to one of the 8 neighbouring cells"
    diag = (ru != rv) & (cu_ != cv_)
    c = g.cost[:, mv].astype(np.int64)
    assert np.array_equal(c[0], np.where(diag, 14, 10)), "distance is the move length"
    speed = 4 - tau
    L = c[0]
    assert np.all(c[1] >= L * speed) and np.all(c[1] <= L * (speed + 2) + 1), "fuel = L (s + 2 h0)"
    for k in range(2, 8):
        assert np.all(c[k] >= L) and np.all(c[k] <= 49 * L // 10 * 10 + 14 * 8 * 9), k
    assert c[10].min() >= 0 and c[10].max() <= 8 * 14
    assert c[11].min() >= 1 and c[11].max() <= 100, "random objective U[1, 100]"
    # a seeded pure function; fewer objectives are a prefix of more
    g2, _ = synth.time_route(1, rows, cols, w, d)
    assert g2.digest() == g.digest()
    g8, _ = synth.time_route(1, rows, cols, w, 8)
    assert np.array_equal(g8.cost, g.cost[:8]) and np.array_equal(g8.col, g.col)
    assert synth.time_route(2, rows, cols, w, d)[0].digest() != g.digest()
