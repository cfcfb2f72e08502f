"""GPU parity at d = 6..8, the objective counts up to OPMOS_MAX_D: single
queries and one batch launch against the oracle, on small random digraphs
with ties and zero-cost arcs. Collected late: these kernel instantiations
are checked after everything else."""
import numpy as np
import pytest

import oracle
import synth
from pins import check_front

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def op():
    import paper_2411_16667_gb300 as pkg
    pkg.build()
    from paper_2411_16667_gb300 import opmos
    if opmos.opmos_device_count() == 0:
        pytest.fail("no CUDA device visible to the library")
    return opmos


@pytest.mark.parametrize("d", [6, 7, 8])
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
