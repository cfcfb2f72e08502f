"""Bounded device-side limits end in an error code the host reads, and the
device stays usable afterwards. Collected last: it sets a process-wide
environment variable (restored when the test ends)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def op():
    import paper_2411_16667_gb300 as pkg
    pkg.build()
    from paper_2411_16667_gb300 import opmos
    if opmos.opmos_device_count() == 0:
        pytest.fail("no CUDA device visible to the library")
    return opmos


def test_time_limit_stops_the_search_with_timeout(op, monkeypatch):
    g, q = synth.config2()
    G = op.opmos_graph.from_synth(g)
    s, t = q[0]
    monkeypatch.setenv("OPMOS_TIME_LIMIT_MS", "1")
    with pytest.raises(op.OpmosError) as e:
        op.opmos_solve(G, s, t, options=op._options(flags=op.FLAG_NO_PATHS))
    assert e.value.code == op.ERR_TIMEOUT
    out = op.opmos_solve_batch(G, [s], [t], mem_budget_bytes=8 << 30)
    assert out[0][0] == op.ERR_TIMEOUT and out[0][1] is None
    monkeypatch.delenv("OPMOS_TIME_LIMIT_MS")
    g1, q1 = synth.config1()
    G1 = op.opmos_graph.from_synth(g1)
    r = op.opmos_solve(G1, *q1[0])
    assert np.array_equal(r.costs, oracle.solve(g1, *q1[0]).costs)
