"""Pins for the sequential NAMOA* oracle (CPU only).

The oracle (Algorithm 1) is checked against facts that do not come from it:
brute-force enumeration (Sec. 3 definition of the cost-unique Pareto set),
textbook Dijkstra (d = 1; per-objective minima; heuristic = ideal point of
Sec. 4), lexicographic Dijkstra, the worked example of Sec. 1, and the
structural invariants of Sec. 3.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from pins import (brute_front, check_front, dijkstra, dominates, lex_dijkstra,
                  load_front_fixture)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tuples(costs):
    return [tuple(int(x) for x in r) for r in costs]


def test_paper_worked_example():
    """Sec. 1: (5,4) and (4,5) are both Pareto-optimal; (6,6) is dominated."""
    arcs, front, n = [], [], 0
    for line in open(os.path.join(GOLDEN, "paper_sec1_two_paths.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "n":
            n = int(f[1])
        elif f[0] == "start":
            s = int(f[1])
        elif f[0] == "goal":
            t = int(f[1])
        elif f[0] == "arc":
            arcs.append((int(f[1]), int(f[2]), (int(f[3]), int(f[4]))))
        elif f[0] == "front":
            front.append((int(f[1]), int(f[2])))
    g = synth.from_arcs(n, arcs)
    res = oracle.solve(g, s, t)
    assert _tuples(res.costs) == sorted(front)
    check_front(g, s, t, res.costs, res.paths)


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random_digraphs(seed):
    """Exact front equals brute-force enumeration on tiny graphs with ties and
    zero-cost arcs (costs in [0,3])."""
    n = 5 + seed % 5
    d = 1 + seed % 5
    g = synth.random_digraph(seed, n, d, p=0.35, cmax=3)
    s, t = 0, n - 1
    expect = brute_front(g, s, t)
    res = oracle.solve(g, s, t)
    assert _tuples(res.costs) == expect
    check_front(g, s, t, res.costs, res.paths)


@pytest.mark.parametrize("d,seed", [(d, seed) for d in range(6, 17) for seed in (301, 304, 306, 308)])
def test_brute_force_high_d(d, seed):
    """The same pin at d = 6..16, the objective counts up to the library's
    maximum (8-node graphs whose fronts hold 6 to 14 vectors)."""
    n = 8
    g = synth.random_digraph(seed, n, d, p=0.45, cmax=3)
    s, t = 0, n - 1
    res = oracle.solve(g, s, t)
    assert _tuples(res.costs) == brute_front(g, s, t)
    check_front(g, s, t, res.costs, res.paths)


@pytest.mark.parametrize("rows,cols,windows,d", [(2, 3, 6, 8), (2, 4, 6, 10), (3, 3, 6, 12), (2, 4, 6, 12),
                                                  (3, 3, 5, 9)])
def test_brute_force_time_routes(rows, cols, windows, d):
    """Brute force on tiny time-expanded ship routes at high d (the routes
    of Sec. 6.1 run up to 12 objectives); the goal is reached through
    zero-cost arcs from every time window of the destination cell."""
    g, q = synth.time_route(3, rows, cols, windows, d)
    s, t = q[0]
    res = oracle.solve(g, s, t)
    assert _tuples(res.costs) == brute_front(g, s, t)
    assert len(res.costs) >= 6
    check_front(g, s, t, res.costs, res.paths)


@pytest.mark.parametrize("rows,cols,d,seed", [(3, 3, 2, 1), (3, 4, 3, 2), (3, 4, 5, 3), (2, 5, 4, 4),
                                              (3, 3, 1, 5), (4, 3, 2, 6)])
def test_brute_force_small_grids(rows, cols, d, seed):
    g = synth.small_grid(seed, rows, cols, d, cmin=0, cmax=4)
    s, t = 0, g.n - 1
    expect = brute_front(g, s, t)
    res = oracle.solve(g, s, t)
    assert _tuples(res.costs) == expect
    check_front(g, s, t, res.costs, res.paths)


@pytest.mark.parametrize("seed", range(6))
def test_single_objective_is_dijkstra(seed):
    """d = 1: the front is the single shortest distance."""
    g = synth.small_grid(seed, 12, 12, 1, cmin=0, cmax=9)
    s, t = 0, g.n - 1
    res = oracle.solve(g, s, t)
    dist = dijkstra(g, s, 0)
    assert _tuples(res.costs) == [(dist[t],)]
    check_front(g, s, t, res.costs, res.paths)


def test_config1_single_objective_projection():
    g, q = synth.config1()
    s, t = q[0]
    g1 = g.first_objectives(1)
    res = oracle.solve(g1, s, t)
    assert _tuples(res.costs) == [(dijkstra(g1, s, 0)[t],)]


def _extreme_point_checks(g, s, t, res):
    costs = res.costs.astype(np.int64)
    for k in range(g.d):
        assert costs[:, k].min() == dijkstra(g, s, k)[t], f"objective {k} minimum"
    assert _tuples(res.costs)[0] == lex_dijkstra(g, s, t)


def test_config1_extreme_points_and_invariants():
    g, q = synth.config1()
    s, t = q[0]
    res = oracle.solve(g, s, t)
    assert len(res.costs) > 10
    _extreme_point_checks(g, s, t, res)
    check_front(g, s, t, res.costs, res.paths)
    # with exact lexicographic extraction and a consistent heuristic no closed
    # label and no solution is ever pruned
    assert res.stats["pruned_closed"] == 0 and res.stats["pruned_p"] == 0


@pytest.mark.parametrize("qi", [0, 2, 3, 5, 7])
def test_config4_queries_extreme_points(qi):
    g, q = synth.config4(1, nq=8)
    s, t = q[qi]
    res = oracle.solve(g, s, t)
    _extreme_point_checks(g, s, t, res)
    check_front(g, s, t, res.costs, res.paths)
    assert res.stats["pruned_closed"] == 0 and res.stats["pruned_p"] == 0


def test_heuristic_is_reverse_dijkstra_and_consistent():
    """Sec. 4 ideal-point heuristic: h_k(v) = shortest v->goal distance."""
    g, q = synth.config1()
    t = q[0][1]
    h = oracle.heuristic(g, t)
    for k in range(g.d):
        ref = dijkstra(g, t, k, reverse=True)
        assert all(int(h[k, v]) == ref[v] for v in range(g.n))
    src = g.src()
    for k in range(g.d):
        assert np.all(h[k, src].astype(np.int64) <= g.cost[k].astype(np.int64) + h[k, g.col])
    assert np.all(h[:, t] == 0)


def test_heuristic_unreachable_is_infinite():
    g = synth.from_arcs(4, [(0, 1, (1, 1)), (1, 2, (1, 1)), (3, 0, (1, 1))])
    h = oracle.heuristic(g, 2)
    assert list(h[0]) == [2, 1, 0, 3]
    h = oracle.heuristic(g, 3)
    assert list(h[0]) == [0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0]


def test_start_equals_goal():
    g = synth.small_grid(3, 3, 3, 2)
    res = oracle.solve(g, 4, 4)
    assert _tuples(res.costs) == [(0, 0)]
    assert list(res.paths[0][0]) == [4] and len(res.paths[0][1]) == 0


def test_unreachable_goal_gives_empty_front():
    g = synth.from_arcs(3, [(0, 1, (1, 2)), (2, 1, (1, 1))])
    res = oracle.solve(g, 0, 2)
    assert res.costs.shape == (0, 2)


def test_zero_cost_cycle_terminates():
    g = synth.from_arcs(3, [(0, 1, (0, 0)), (1, 0, (0, 0)), (1, 2, (1, 0)), (0, 2, (0, 1))])
    res = oracle.solve(g, 0, 2)
    assert _tuples(res.costs) == [(0, 1), (1, 0)]


def test_label_budget_and_overflow_are_reported():
    g, q = synth.config1()
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve(g, *q[0], label_budget=100)
    assert e.value.code == oracle.BUDGET
    big = synth.from_arcs(3, [(0, 1, (0xF0000000,)), (1, 2, (0xF0000000,))])
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve(big, 0, 2)
    assert e.value.code == oracle.OVERFLOW


def test_invalid_arguments():
    g = synth.small_grid(1, 2, 2, 2)
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve(g, 0, 99)
    assert e.value.code == oracle.INVALID


def test_golden_fixtures_are_self_consistent():
    """Every committed oracle front fixture is cost-unique and non-dominated."""
    for name in sorted(os.listdir(GOLDEN)):
        if not name.endswith(".front"):
            continue
        meta, costs = load_front_fixture(os.path.join(GOLDEN, name))
        assert costs.shape[0] == meta["count"]
        vecs = _tuples(costs)
        assert vecs == sorted(set(vecs))
        arr = costs.astype(np.int64)
        for i in range(arr.shape[0]):
            le = np.all(arr <= arr[i], axis=1) & np.any(arr < arr[i], axis=1)
            assert not le.any(), f"{name}: row {i} dominated"


def test_dominance_helper_definition():
    assert dominates((4, 5), (5, 5)) and not dominates((5, 5), (5, 5))
    assert not dominates((4, 6), (5, 5))
