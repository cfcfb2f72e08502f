"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Fronts are compared bit-exactly as sets of uint32 cost vectors; every GPU
path is re-verified (valid arcs, cost sum equals its vector). Paths are not
compared with the oracle's, because several paths can carry the same cost.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from pins import check_front, check_front_sampled, load_front_fixture

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def op():
    import paper_2411_16667_gb300 as pkg
    pkg.build()
    from paper_2411_16667_gb300 import opmos
    if opmos.opmos_device_count() == 0:
        pytest.fail("no CUDA device visible to the library")
    return opmos


def _same_front(res, expect: np.ndarray):
    got = res.costs
    assert got.shape == expect.shape, f"front size {got.shape[0]} != oracle {expect.shape[0]}"
    assert np.array_equal(got, expect), "front differs from the oracle"


# ---------------------------------------------------------------------------
# heuristic (Sec. 4 ideal point) -- bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("maker", ["config1", "ship64", "rand"])
def test_heuristic_matches_oracle(op, maker):
    if maker == "config1":
        g, q = synth.config1()
    elif maker == "ship64":
        g, q = synth.ship_grid(3, 64, 5)
    else:
        g = synth.random_digraph(11, 40, 3, p=0.08, cmax=9)
        q = [(0, 7)]
    goal = q[0][1]
    G = op.opmos_graph.from_synth(g)
    h = op.opmos_heur(G, goal).copy()
    assert np.array_equal(h, oracle.heuristic(g, goal))


def test_heuristic_full_size_ship_grid(op):
    g, q = synth.config2()
    G = op.opmos_graph.from_synth(g)
    h = op.opmos_heur(G, q[0][1]).copy()
    assert np.array_equal(h, oracle.heuristic(g, q[0][1]))


# ---------------------------------------------------------------------------
# single-query search -- bit-exact fronts
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(24))
def test_random_digraphs(op, seed):
    n = 5 + seed % 7
    d = 1 + seed % 5
    g = synth.random_digraph(seed, n, d, p=0.35, cmax=3)
    s, t = 0, n - 1
    exp = oracle.solve(g, s, t)
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, s, t, window=1 + seed % 5)
    _same_front(res, exp.costs)
    check_front(g, s, t, res.costs, res.paths)


def test_config1_front(op):
    g, q = synth.config1()
    s, t = q[0]
    exp = oracle.solve(g, s, t)
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, s, t)
    _same_front(res, exp.costs)
    check_front(g, s, t, res.costs, res.paths)
    assert res.stats["extracted"] >= 1 and res.stats["steps"] >= 1


@pytest.mark.parametrize("rows,d,seed", [(48, 3, 1), (64, 3, 2), (96, 3, 3), (64, 5, 4), (40, 2, 5), (33, 4, 6)])
def test_ship_grids(op, rows, d, seed):
    """Sizes span many frontier tiles with ragged tails and several windows."""
    g, q = synth.ship_grid(seed, rows, d)
    s, t = q[0]
    exp = oracle.solve(g, s, t)
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, s, t)
    _same_front(res, exp.costs)
    check_front(g, s, t, res.costs, res.paths)


@pytest.mark.parametrize("window,lanes,tile,delta", [(1, 4, 32, 1), (7, 16, 64, 1), (64, 32, 32, 3),
                                                     (100000, 8, 128, 1), (512, 8, 32, 50)])
def test_launch_parameters_do_not_change_the_front(op, window, lanes, tile, delta):
    g, q = synth.ship_grid(7, 48, 3)
    s, t = q[0]
    exp = oracle.solve(g, s, t)
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, s, t, window=window, lanes_per_label=lanes, tile=tile, delta=delta)
    _same_front(res, exp.costs)
    check_front(g, s, t, res.costs, res.paths)


def test_d_used_prefix_of_objectives(op):
    g, q = synth.ship_grid(8, 48, 5)
    s, t = q[0]
    G = op.opmos_graph.from_synth(g)
    for d in (1, 2, 4):
        exp = oracle.solve(g.first_objectives(d), s, t)
        res = op.opmos_solve(G, s, t, d_used=d)
        _same_front(res, exp.costs)


def test_given_heuristic_is_used(op):
    g, q = synth.config1()
    s, t = q[0]
    G = op.opmos_graph.from_synth(g)
    H = op.opmos_heur(G, t)
    res = op.opmos_solve(G, s, t, heur=H)
    _same_front(res, oracle.solve(g, s, t).costs)
    assert res.stats["heuristic_ns"] == 0


@pytest.mark.parametrize("window", [1024, 262144])
def test_config2_full_size_against_golden(op, window):
    """Full 256x256 3-objective ship grid against the committed oracle front,
    with the default window (one 512-thread block per SM) and the large
    window the bench picks (three 256-thread blocks per SM, split merges)."""
    meta, expect = load_front_fixture(os.path.join(GOLDEN, "config2_seed1_q0.front"))
    g, q = synth.config2()
    if g.digest() != meta["digest"]:
        pytest.fail(f"regenerated graph digest {g.digest()} != fixture {meta['digest']}")
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, meta["start"], meta["goal"], window=window)
    _same_front(res, expect)
    # the front equals the oracle's bit for bit; every path is re-verified
    check_front_sampled(g, meta["start"], meta["goal"], res.costs, res.paths, nrows=500,
                        npaths=len(res.paths))


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------
def test_start_equals_goal(op):
    g = synth.small_grid(1, 4, 4, 3)
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, 5, 5)
    assert res.costs.tolist() == [[0, 0, 0]]
    assert res.paths[0][0].tolist() == [5] and res.paths[0][1].size == 0


def test_unreachable_goal(op):
    g = synth.from_arcs(3, [(0, 1, (1, 2)), (2, 1, (1, 1))])
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, 0, 2)
    assert res.costs.shape == (0, 2)


def test_zero_cost_cycles_and_ties(op):
    g = synth.from_arcs(3, [(0, 1, (0, 0)), (1, 0, (0, 0)), (1, 2, (1, 0)), (0, 2, (0, 1))])
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, 0, 2)
    assert res.costs.tolist() == [[0, 1], [1, 0]]
    check_front(g, 0, 2, res.costs, res.paths)


def test_no_paths_flag(op):
    g, q = synth.config1()
    G = op.opmos_graph.from_synth(g)
    res = op.opmos_solve(G, *q[0], flags=op.FLAG_NO_PATHS)
    assert res.paths is None
    _same_front(res, oracle.solve(g, *q[0]).costs)


def test_label_budget_is_reported(op):
    g, q = synth.config1()
    G = op.opmos_graph.from_synth(g)
    with pytest.raises(op.OpmosError) as e:
        op.opmos_solve(G, *q[0], label_budget=50)
    assert e.value.code == op.ERR_BUDGET
    # the library is usable afterwards
    _same_front(op.opmos_solve(G, *q[0]), oracle.solve(g, *q[0]).costs)


def test_small_arena_is_capacity_error(op):
    g, q = synth.ship_grid(2, 96, 3)
    G = op.opmos_graph.from_synth(g)
    with pytest.raises(op.OpmosError) as e:
        op.opmos_solve(G, *q[0], mem_budget_bytes=10 << 20, window=64)
    assert e.value.code == op.ERR_CAPACITY


def test_invalid_arguments(op):
    g, q = synth.config1()
    G = op.opmos_graph.from_synth(g)
    for kw in ({"lanes_per_label": 3}, {"tile": 48}, {"d_used": 3}):
        with pytest.raises(op.OpmosError) as e:
            op.opmos_solve(G, *q[0], **kw)
        assert e.value.code == op.ERR_INVALID_ARG
    with pytest.raises(op.OpmosError) as e:
        op.opmos_solve(G, 0, 5000)
    assert e.value.code == op.ERR_INVALID_ARG
    bad = synth.from_arcs(3, [(0, 1, (0xF0000000,)), (1, 2, (1,))])
    with pytest.raises(op.OpmosError) as e:
        op.opmos_graph.from_synth(bad)
    assert e.value.code == op.ERR_OVERFLOW


# ---------------------------------------------------------------------------
# batch mode
# ---------------------------------------------------------------------------
def _digest(costs) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(costs, dtype="<u4").tobytes()).hexdigest()[:16]


def test_config4_full_batch_against_oracle_digests(op):
    """All 1,024 queries of the 5-objective ship grid in one batch: every
    front the oracle finished within its label budget matches its committed
    digest; the others satisfy the Sec. 3 invariants and the ideal point."""
    rows = [line.split() for line in open(os.path.join(GOLDEN, "config4_seed1.digests"))
            if line.strip() and not line.startswith("#")]
    graph_line, rows = rows[0], rows[1:]
    g, queries = synth.config4(1)
    assert graph_line[2] == g.digest(), "regenerated graph does not match the digest file"
    G = op.opmos_graph.from_synth(g)
    out = op.opmos_solve_batch(G, [s for s, _ in queries], [t for _, t in queries])
    unchecked = 0
    for (qi, s, t, count, _labels, _ext, dig), (st, res) in zip(rows, out):
        s, t = int(s), int(t)
        assert (s, t) == queries[int(qi)]
        assert st == op.OK, f"query {qi} status {st}"
        if int(count) >= 0:
            assert res.costs.shape[0] == int(count), f"query {qi}: {res.costs.shape[0]} != {count}"
            assert _digest(res.costs) == dig, f"query {qi}: front differs from the oracle"
        else:
            unchecked += 1
            check_front_sampled(g, s, t, res.costs, res.paths)
            h = oracle.heuristic(g, t)
            assert np.array_equal(res.costs.min(axis=0), h[:, s])
    assert unchecked == sum(1 for r in rows if int(r[3]) < 0)


def test_batch_matches_oracle_on_small_ship_queries(op):
    g, queries = synth.config4(1, nq=48)
    rows = [line.split() for line in open(os.path.join(GOLDEN, "config4_seed1.digests"))
            if line.strip() and not line.startswith("#")][1:49]
    small = [int(r[0]) for r in rows if 0 <= int(r[4]) <= 60000][:24]
    G = op.opmos_graph.from_synth(g)
    qs = [queries[i] for i in small]
    out = op.opmos_solve_batch(G, [s for s, _ in qs], [t for _, t in qs], window=64)
    for (s, t), (st, res) in zip(qs, out):
        assert st == op.OK, f"query {s}->{t} status {st}"
        exp = oracle.solve(g, s, t)
        _same_front(res, exp.costs)
        check_front(g, s, t, res.costs, res.paths)


def _same_paths(a, b):
    assert len(a.paths) == len(b.paths)
    for (na, ea), (nb, eb) in zip(a.paths, b.paths):
        assert np.array_equal(na, nb) and np.array_equal(ea, eb)


def test_batch_equals_single(op):
    """Each query's result -- front and the path kept for every cost -- is
    the same alone and in the batch, given the same launch parameters (ties
    between equal-cost candidates go to the smallest arc id; a label pruned
    in a step is still extractable in it, so the windows do not depend on
    thread timing)."""
    g, queries = synth.config4(2, nq=12)
    G = op.opmos_graph.from_synth(g)
    out = op.opmos_solve_batch(G, [s for s, _ in queries], [t for _, t in queries], window=64)
    for (s, t), (st, res) in zip(queries, out):
        assert st == op.OK
        alone = op.opmos_solve(G, s, t, window=64)
        assert np.array_equal(res.costs, alone.costs)
        _same_paths(res, alone)
        check_front(g, s, t, res.costs, res.paths)


def test_paths_repeat_exactly(op):
    """Three runs of the same query, single and batched, keep the same path
    for every cost (SURVEY reading c5: several paths may carry one cost; the
    library's choice is deterministic)."""
    g, q = synth.ship_grid(9, 96, 3)
    s, t = q[0]
    G = op.opmos_graph.from_synth(g)
    runs = [op.opmos_solve(G, s, t, window=256) for _ in range(3)]
    runs += [op.opmos_solve_batch(G, [s, 0], [t, 5000], window=256)[0][1]]
    for r in runs[1:]:
        assert np.array_equal(r.costs, runs[0].costs)
        _same_paths(r, runs[0])
    # the wide grid (large windows): repeated runs keep their paths too
    wide = [op.opmos_solve(G, s, t, window=65536) for _ in range(3)]
    for r in wide[1:]:
        assert np.array_equal(r.costs, runs[0].costs)
        _same_paths(r, wide[0])


def test_batch_graph_capture_gives_the_same_fronts(op):
    """OPMOS_FLAG_GRAPH: the launch captured into a CUDA graph and replayed."""
    g, queries = synth.config4(2, nq=16)
    G = op.opmos_graph.from_synth(g)
    starts, goals = [s for s, _ in queries], [t for _, t in queries]
    plain = op.opmos_solve_batch(G, starts, goals, window=128)
    captured = op.opmos_solve_batch(G, starts, goals, window=128, flags=op.FLAG_GRAPH)
    for (s, t), (sa, ra), (sb, rb) in zip(queries, plain, captured):
        assert sa == sb == op.OK
        assert np.array_equal(ra.costs, rb.costs)
        check_front(g, s, t, rb.costs, rb.paths)


def test_batch_with_duplicate_and_trivial_queries(op):
    g, q = synth.config1()
    G = op.opmos_graph.from_synth(g)
    s, t = q[0]
    out = op.opmos_solve_batch(G, [s, s, t, 5], [t, t, t, 900])
    exp = oracle.solve(g, s, t).costs
    assert out[0][0] == op.OK and np.array_equal(out[0][1].costs, exp)
    assert np.array_equal(out[1][1].costs, exp)
    assert out[2][1].costs.tolist() == [[0, 0]]
    _same_front(out[3][1], oracle.solve(g, 5, 900).costs)


# ---------------------------------------------------------------------------
# config 3: 200k-node road-like graph, 4 objectives
# ---------------------------------------------------------------------------
def test_config3_road_graph_against_oracle(op):
    """Every query among the first 16 that the oracle finishes within 300k
    labels on the first two objectives, plus query 4 on the first three; each
    alone and all together in one batch launch. (At d=4 the probed queries
    exceed any label budget the oracle can meet in a test.)"""
    g, queries = synth.config3()
    G = op.opmos_graph.from_synth(g)
    cases = []
    for d, idx in ((2, range(16)), (3, [4])):
        gd = g.first_objectives(d)
        for i in idx:
            s, t = queries[i]
            f = oracle.solve(gd, s, t, label_budget=300_000, partial_ok=True)
            if not f.stats["partial"]:
                cases.append((d, s, t, f.costs))
    assert sum(1 for c in cases if c[0] == 2) >= 4 and any(c[0] == 3 for c in cases)
    for d, s, t, exp in cases:
        res = op.opmos_solve(G, s, t, d_used=d)
        _same_front(res, exp)
        check_front(g.first_objectives(d), s, t, res.costs, res.paths)
    two = [c for c in cases if c[0] == 2]
    out = op.opmos_solve_batch(G, [c[1] for c in two], [c[2] for c in two], d_used=2)
    for (d, s, t, exp), (st, res) in zip(two, out):
        assert st == op.OK, f"query {s}->{t} status {st}"
        _same_front(res, exp)


def test_config3_full_d_against_oracle_digests(op):
    """Config 3 at its full d=4: all 8 fewest-hop queries, whose oracle fronts
    (22.5k to 59k solutions) are committed as digests, in one batch launch,
    and the three cheapest alone."""
    rows = [line.split() for line in open(os.path.join(GOLDEN, "config3_seed1_short8.digests"))
            if line.strip() and not line.startswith("#")]
    graph_line, rows = rows[0], rows[1:]
    g, queries = synth.config3()
    assert graph_line[2] == g.digest(), "regenerated graph does not match the digest file"
    done = sorted((r for r in rows if int(r[3]) >= 0), key=lambda r: int(r[5]))
    assert len(done) == 8
    G = op.opmos_graph.from_synth(g)
    starts, goals = [int(r[1]) for r in done], [int(r[2]) for r in done]
    out = op.opmos_solve_batch(G, starts, goals)
    for r, s, t, (st, res) in zip(done, starts, goals, out):
        assert (s, t) == queries[int(r[0])]
        assert st == op.OK, f"query {r[0]} status {st}"
        assert res.costs.shape[0] == int(r[3]), f"query {r[0]}: {res.costs.shape[0]} != {r[3]}"
        assert _digest(res.costs) == r[6], f"query {r[0]}: front differs from the oracle"
        check_front_sampled(g, s, t, res.costs, res.paths)
    for r, s, t in list(zip(done, starts, goals))[:3]:
        alone = op.opmos_solve(G, s, t, options=op._options(flags=op.FLAG_NO_PATHS))
        assert _digest(alone.costs) == r[6], f"query {r[0]} alone: front differs from the oracle"


def test_config3_full_d_batch_under_label_budget(op):
    """All four objectives, 32 queries in one launch with a per-query label
    budget (the time-limit practice of Sec. 6.1): each query ends OK with a
    valid front or is reported as over budget; none fails otherwise."""
    g, queries = synth.config3()
    G = op.opmos_graph.from_synth(g)
    qs = queries[:32]
    out = op.opmos_solve_batch(G, [s for s, _ in qs], [t for _, t in qs], label_budget=200_000)
    assert len(out) == len(qs)
    for (s, t), (st, res) in zip(qs, out):
        assert st in (op.OK, op.ERR_BUDGET), f"query {s}->{t} status {st}"
        if st == op.OK:
            check_front_sampled(g, s, t, res.costs, res.paths)


# ---------------------------------------------------------------------------
# FIFO (relaxed-order) OPEN: Sec. 4 and 7.1 compare it with the priority queue
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("window", [1, 64, 1024])
def test_fifo_order_gives_the_same_front(op, window):
    """OPMOS_FLAG_FIFO takes the oldest OPEN entries each step instead of the
    lexicographically lowest: the front is the same, only the work differs."""
    cases = [synth.config1(), synth.ship_grid(3, 48, 3), (synth.random_digraph(5, 9, 4, p=0.35, cmax=3), [(0, 8)])]
    for g, q in cases:
        s, t = q[0]
        G = op.opmos_graph.from_synth(g)
        exp = oracle.solve(g, s, t)
        res = op.opmos_solve(G, s, t, window=window, flags=op.FLAG_FIFO)
        _same_front(res, exp.costs)
        check_front(g, s, t, res.costs, res.paths)


def test_fifo_batch_and_work_ratio(op):
    """FIFO in a batch launch gives the oracle's fronts; on the 48x48 ship
    grid it extracts more labels than the ordered window of the same width
    (the work inefficiency of Sec. 4)."""
    g, queries = synth.config4(2, nq=12)
    G = op.opmos_graph.from_synth(g)
    starts, goals = [s for s, _ in queries], [t for _, t in queries]
    out = op.opmos_solve_batch(G, starts, goals, window=256, flags=op.FLAG_FIFO)
    for (s, t), (st, res) in zip(queries, out):
        assert st == op.OK
        _same_front(res, op.opmos_solve(G, s, t, window=256).costs)
    g2, q2 = synth.ship_grid(3, 48, 3)
    G2 = op.opmos_graph.from_synth(g2)
    ordered = op.opmos_solve(G2, *q2[0], window=256)
    fifo = op.opmos_solve(G2, *q2[0], window=256, flags=op.FLAG_FIFO)
    assert fifo.stats["extracted"] > ordered.stats["extracted"]
