"""GPU parity at high objective counts against the oracle: d = 6..16 (the
library's maximum) on small random digraphs with ties and zero-cost arcs,
and time-expanded ship routes at d = 8, 10 and 12 (the regime of the paper's
routes, Sec. 6.1, where label processing dominates, Sec. 4). Single queries
and batch launches. Collected late: these kernel instantiations are checked
after everything else."""
import numpy as np
import pytest

import oracle
import synth
from pins import check_front, check_front_sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def op():
    import paper_2411_16667_gb300 as pkg
    pkg.build()
    from paper_2411_16667_gb300 import opmos
    if opmos.opmos_device_count() == 0:
        pytest.fail("no CUDA device visible to the library")
    return opmos


@pytest.mark.parametrize("d", list(range(6, 17)))
def test_high_d_single_and_batch(op, d):
    graphs = [synth.random_digraph(seed, 8, d, p=0.45, cmax=3) for seed in (301, 304, 306, 308)]
    for g in graphs:
        exp = oracle.solve(g, 0, 7)
        G = op.opmos_graph.from_synth(g)
        res = op.opmos_solve(G, 0, 7)
        assert np.array_equal(res.costs, exp.costs)
        check_front(g, 0, 7, res.costs, res.paths)
    g = graphs[1]
    G = op.opmos_graph.from_synth(g)
    qs = [(0, 7), (1, 6), (2, 5), (3, 7), (0, 0)]
    out = op.opmos_solve_batch(G, [s for s, _ in qs], [t for _, t in qs], mem_budget_bytes=4 << 30)
    for (s, t), (st, res) in zip(qs, out):
        assert st == op.OK
        assert np.array_equal(res.costs, oracle.solve(g, s, t).costs)
        check_front(g, s, t, res.costs, res.paths)


def _route_queries(g, rows, cols, windows):
    """The route's own query plus departures from other cells in window 0."""
    goal = rows * cols * windows
    cells = [0, 1, cols, cols + 1, 2 * cols]
    return [(c * windows, goal) for c in cells if c < rows * cols - 1]


@pytest.mark.parametrize("d", [8, 10, 12])
def test_time_routes_against_oracle(op, d):
    rows, cols, windows = 4, 5, 10
    for seed in (1, 2):
        g, _ = synth.time_route(seed, rows, cols, windows, d)
        G = op.opmos_graph.from_synth(g)
        qs = _route_queries(g, rows, cols, windows)
        exp = [oracle.solve(g, s, t).costs for s, t in qs]
        assert len(exp[0]) >= 50
        res = op.opmos_solve(G, *qs[0])
        assert np.array_equal(res.costs, exp[0])
        check_front(g, *qs[0], res.costs, res.paths)
        out = op.opmos_solve_batch(G, [s for s, _ in qs], [t for _, t in qs], mem_budget_bytes=8 << 30)
        for (s, t), e, (st, r) in zip(qs, exp, out):
            assert st == op.OK, f"query {s}->{t} status {st}"
            assert np.array_equal(r.costs, e)
            check_front(g, s, t, r.costs, r.paths)


def test_time_route_d12_large_front(op):
    """A d = 12 route whose front holds about 1,800 vectors (frontiers past
    the block-merge threshold): single query, default, small and large
    windows."""
    g, q = synth.time_route(1, 4, 6, 16, 12)
    s, t = q[0]
    exp = oracle.solve(g, s, t)
    assert len(exp.costs) > 1000
    G = op.opmos_graph.from_synth(g)
    for w in (1024, 64, 16384):  # the last one on the wide grid
        res = op.opmos_solve(G, s, t, window=w)
        assert np.array_equal(res.costs, exp.costs)
    check_front(g, s, t, res.costs, res.paths)


def test_time_routes_against_oracle_digests(op):
    """The committed oracle digests of four time-expanded routes, up to the
    d = 12 route whose front holds 16,268 vectors (tests/golden/routes.digests,
    written by tests/golden/make_golden.py routes)."""
    import hashlib
    import os
    rows = [line.split() for line in open(os.path.join(os.path.dirname(__file__), "golden", "routes.digests"))
            if line.strip() and not line.startswith("#")]
    assert len(rows) == 4
    for name, gdig, s, t, count, _labels, _ext, fdig in rows:
        dims = name.split("-")[0][len("route"):].split("x")
        d = int(name.split("-d")[1].split("-")[0])
        seed = int(name.split("-s")[-1])
        g, q = synth.time_route(seed, int(dims[0]), int(dims[1]), int(dims[2]), d)
        assert g.name == name and g.digest() == gdig and q[0] == (int(s), int(t))
        G = op.opmos_graph.from_synth(g)
        res = op.opmos_solve(G, int(s), int(t))
        assert res.costs.shape[0] == int(count), f"{name}: {res.costs.shape[0]} != {count}"
        got = hashlib.sha256(np.ascontiguousarray(res.costs, dtype="<u4").tobytes()).hexdigest()[:16]
        assert got == fdig, f"{name}: front differs from the oracle"
        check_front_sampled(g, int(s), int(t), res.costs, res.paths, nrows=400, npaths=200)
