"""Serving: continuous batching through opmos_server_* (C ABI).

Queries over several device-resident graphs with different objective counts
are submitted while earlier ones are still running; every front must equal
the same query solved alone (and the oracle's), and every path must verify.
"""
import time

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


def _wait(op, srv, tickets, timeout=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t in done:
                continue
            st, r = srv.poll(t)
            if st != op.PENDING:
                done[t] = (st, r)
        time.sleep(0.001)
    assert len(done) == len(tickets), "server did not finish in time"
    return done


def test_server_mixed_graphs_and_objective_counts(op):
    g1, q1 = synth.config1()
    g2, q2 = synth.ship_grid(5, 40, 5)
    g3 = synth.random_digraph(9, 30, 3, p=0.12, cmax=6)
    graphs = [g1, g2, g3]
    G = [op.opmos_graph.from_synth(g) for g in graphs]
    rng = np.random.default_rng(3)
    plan = []
    for i in range(36):
        gi = int(rng.integers(0, 3))
        g = graphs[gi]
        d = int(rng.integers(1, g.d + 1))
        s, t = (int(x) for x in rng.integers(0, g.n, size=2))
        plan.append((gi, d, s, t))
    # each query alone, before the server makes its kernel resident (other
    # compute entry points must not run beside a resident server kernel)
    alone = [op.opmos_solve(G[gi], s, t, d_used=d, window=64) for gi, d, s, t in plan]
    srv = op.opmos_server(G, mem_budget_bytes=8 << 30, window=64)
    first = [srv.submit(*p) for p in plan[:18]]
    time.sleep(0.01)  # the rest arrives while the first ones run
    rest = [srv.submit(*p) for p in plan[18:]]
    results = _wait(op, srv, first + rest)
    srv.close()
    for ticket, (gi, d, s, t), ref in zip(first + rest, plan, alone):
        st, r = results[ticket]
        assert st == op.OK, f"query {(gi, d, s, t)} status {st}"
        gd = graphs[gi].first_objectives(d)
        assert np.array_equal(r.costs, ref.costs)
        assert len(r.paths) == len(ref.paths)
        for (na, ea), (nb, eb) in zip(r.paths, ref.paths):  # the same path for every cost
            assert np.array_equal(na, nb) and np.array_equal(ea, eb)
        assert np.array_equal(r.costs, oracle.solve(gd, s, t).costs)
        check_front(gd, s, t, r.costs, r.paths)


def test_server_queue_full_is_reported(op):
    g, q = synth.config1()
    G = op.opmos_graph.from_synth(g)
    srv = op.opmos_server([G], mem_budget_bytes=2 << 30)
    tickets = []
    with pytest.raises(op.OpmosError) as e:
        for _ in range(100000):
            tickets.append(srv.submit(0, 2, 0, 1023))
    assert e.value.code == op.ERR_CAPACITY
    res = _wait(op, srv, tickets)
    exp = oracle.solve(g, 0, 1023).costs
    assert all(st == op.OK and np.array_equal(r.costs, exp) for st, r in res.values())
    # after collecting, the queue accepts again
    t = srv.submit(0, 1, 5, 900)
    st, r = _wait(op, srv, [t])[t]
    assert st == op.OK and np.array_equal(r.costs, oracle.solve(g.first_objectives(1), 5, 900).costs)
    srv.close()
