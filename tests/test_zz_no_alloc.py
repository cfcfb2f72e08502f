"""The allocation-free heuristic entry point against the allocating one.

opmos_heuristic_noalloc serves callers that cannot allocate device memory
while they run (their memory is all reserved by their own pool, or they must
not pay for cudaMalloc's cost and synchronisation). The caller owns the output
buffer -- here a torch tensor -- and the call uses only a fixed scratch array
inside the library. Two calls in a row must both match opmos_heuristic
exactly (integer distances), the second reusing the scratch left by the
first. This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def _noalloc(op, G, goal, d):
    import torch
    out = torch.full((d or G.d, G.n), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    op.opmos_heuristic_noalloc(G, goal, d, out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_noalloc_matches_allocating_heuristic_twice(op):
    g, q = synth.ship_grid(4, 96, 5)
    G = op.opmos_graph.from_synth(g)
    goals = [q[0][1], 17]
    for goal in goals:  # two calls in a row on the shared scratch
        ref = op.opmos_heur(G, goal).copy()
        got = _noalloc(op, G, goal, 0)
        assert np.array_equal(got, ref)


def test_noalloc_allocates_no_device_memory(op):
    """The property the entry point exists for: after a warm-up call (the
    one-time address lookup, module loading), further calls leave the
    device's free memory unchanged."""
    import torch
    g, q = synth.ship_grid(4, 96, 5)
    G = op.opmos_graph.from_synth(g)
    out = torch.empty((g.d, g.n), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    op.opmos_heuristic_noalloc(G, q[0][1], 0, out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for goal in (q[0][1], 5, 17):
        op.opmos_heuristic_noalloc(G, goal, 0, out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, f"free device memory dropped by {free0 - free1} bytes"


def test_noalloc_first_objectives_and_small_graph(op):
    g, q = synth.config1()
    G = op.opmos_graph.from_synth(g)
    ref = op.opmos_heur(G, q[0][1], 1).copy()
    for _ in range(2):
        assert np.array_equal(_noalloc(op, G, q[0][1], 1), ref)


def test_noalloc_rejects_graphs_beyond_its_limit(op):
    n = (1 << 18) + 5
    arcs = [(i, i + 1, (1,)) for i in range(n - 1)]
    g = synth.from_arcs(n, arcs)
    G = op.opmos_graph.from_synth(g)
    import torch
    out = torch.empty((1, n), dtype=torch.int32, device="cuda")
    with pytest.raises(op.OpmosError) as e:
        op.opmos_heuristic_noalloc(G, 0, 1, out.data_ptr())
    assert e.value.code == op.ERR_CAPACITY
    assert "at most" in str(e.value)
