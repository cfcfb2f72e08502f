"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
round-robin split of independent queries over ranks, the max-over-ranks
timing, and the reference arm under torchrun (rank 0 alone reports)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_queries(10, rank, world)
        est = [5, 1, 9, 9, 2, 7, 3, 3, 8, 0]
        by_cost = bench.shard_queries(10, rank, world, est)
        m = bench.max_over_ranks(float(10 * (rank + 1)), device="cpu")
        bench.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"mine": mine, "max": m, "by_cost": by_cost}, f)
    finally:
        dist.destroy_process_group()


def test_shards_are_disjoint_and_max_is_global(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    allq = sorted(q for r in res for q in r["mine"])
    assert allq == list(range(10))
    assert not set(res[0]["mine"]) & set(res[1]["mine"])
    assert all(r["max"] == 20.0 for r in res)
    # by estimated cost: disjoint, complete, and the two ranks' totals within the largest single cost
    est = [5, 1, 9, 9, 2, 7, 3, 3, 8, 0]
    assert sorted(q for r in res for q in r["by_cost"]) == list(range(10))
    tot = [sum(est[i] for i in r["by_cost"]) for r in res]
    assert abs(tot[0] - tot[1]) <= max(est)
    assert {2, 3} <= set(res[0]["by_cost"]) | set(res[1]["by_cost"])
    assert not ({2, 3} <= set(res[0]["by_cost"])), "the two most expensive queries go to different ranks"


def test_single_process_helpers_without_a_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard_queries(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.max_over_ranks(3.5, device="cpu") == 3.5


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--cpu-labels", "20000"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
