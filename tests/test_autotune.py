"""Autotuner logic (CPU, fake solver) and on the GPU (real solves)."""
import json

import numpy as np
import pytest

import synth
from paper_2411_16667_gb300 import autotune, opmos


class _FakeGraph:
    def __init__(self, g):
        self.n, self.d, self.rowptr, self.col, self.cost = g.n, g.d, g.rowptr, g.col, g.cost.reshape(-1)


def _fake(monkeypatch, front_of):
    class R:
        def __init__(self, costs, ns):
            self.costs = costs
            self.stats = {"search_ns": ns}

    def solve(graph, s, t, heur=None, options=None):
        return R(front_of(options), 1000 * options.window + 10 * options.lanes_per_label + options.tile)

    monkeypatch.setattr(opmos, "opmos_solve", solve)
    monkeypatch.setattr(opmos, "opmos_heur", lambda *a, **k: None)


def test_picks_fastest_and_caches(monkeypatch, tmp_path):
    g = _FakeGraph(synth.small_grid(1, 3, 3, 2))
    _fake(monkeypatch, lambda o: np.array([[1, 2]], np.uint32))
    autotune._cache.clear()
    path = str(tmp_path / "tune.json")
    ch = autotune.autotune(g, [(0, 8)], windows=(64, 32), lanes=(8, 4), tiles=(64, 32), cache_path=path)
    assert (ch.window, ch.lanes_per_label, ch.tile) == (32, 4, 32)
    assert len(ch.table) == 8
    disk = json.load(open(path))
    assert list(disk.values())[0]["window"] == 32
    autotune._cache.clear()
    _fake(monkeypatch, lambda o: (_ for _ in ()).throw(AssertionError("cache not used")))
    again = autotune.autotune(g, [(0, 8)], cache_path=path)
    assert (again.window, again.lanes_per_label, again.tile) == (32, 4, 32)


def test_a_configuration_that_changes_the_front_is_an_error(monkeypatch):
    g = _FakeGraph(synth.small_grid(2, 3, 3, 2))
    _fake(monkeypatch, lambda o: np.array([[o.window, 0]], np.uint32))
    autotune._cache.clear()
    with pytest.raises(RuntimeError):
        autotune.autotune(g, [(0, 8)], windows=(64, 32), lanes=(8,), tiles=(32,))


@pytest.mark.gpu
def test_autotune_on_the_gpu_keeps_the_front():
    import oracle
    import paper_2411_16667_gb300 as pkg
    pkg.build()
    g, q = synth.ship_grid(3, 40, 3)
    G = opmos.opmos_graph.from_synth(g)
    autotune._cache.clear()
    ch = autotune.autotune(G, q, windows=(64, 512), lanes=(8, 16), tiles=(32,))
    assert len(ch.table) == 4
    res = opmos.opmos_solve(G, *q[0], options=ch.options())
    assert np.array_equal(res.costs, oracle.solve(g, *q[0]).costs)
    gb, qb = synth.config4(2, nq=6)
    Gb = opmos.opmos_graph.from_synth(gb)
    chb = autotune.autotune(Gb, qb, mode="batch", windows=(64, 256), lanes=(8,), tiles=(32,))
    assert chb.window in (64, 256)
