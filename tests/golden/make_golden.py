"""Write oracle fronts for full-size synthetic workloads as text fixtures.

Usage: python tests/golden/make_golden.py config2 [--seed 1]
       python tests/golden/make_golden.py config4 --digests --jobs 6
       python tests/golden/make_golden.py config3 --digests --shortest-hops 8 \
              --budget 5000000 --jobs 8
       python tests/golden/make_golden.py routes --jobs 4

Only the oracle (Algorithm 1, ``oracle/``) and the input generators
(``synth``) are called. Each fixture records the graph digest so a test can
tell whether the graph it regenerated is the one the front belongs to.

File format (one fixture per query):
    # <free text>
    graph <name> <digest>
    query <start> <goal>
    d <d>
    stats <key>=<value> ...
    count <k>
    <c_0> <c_1> ... <c_{d-1}>      (k lines, lexicographic order)

Digest format (``--digests``; one line per query of the config):
    <qi> <start> <goal> <count> <labels> <extracted> <sha256 of the sorted
    front as little-endian uint32, first 16 hex digits>
A query the oracle cannot finish within ``--budget`` labels is written with
count -1.

Route digests (``routes``; time-expanded ship routes of ``synth.time_route``,
one line per instance in ROUTES):
    <name> <graph digest> <start> <goal> <count> <labels> <extracted> <sha256[:16]> ``--shortest-hops K`` restricts the digests to the K queries with
the fewest hops between start and goal (breadth-first search, ties by query
index): the queries most likely to finish at full d.
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time

_ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write_front(path, g, s, t, front, note=""):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write(f"# oracle front (Algorithm 1, sequential NAMOA*) {note}\n")
        f.write(f"graph {g.name} {g.digest()}\n")
        f.write(f"query {s} {t}\n")
        f.write(f"d {g.d}\n")
        f.write("stats " + " ".join(f"{k}={v}" for k, v in front.stats.items()) + "\n")
        f.write(f"count {len(front.costs)}\n")
        for row in front.costs:
            f.write(" ".join(str(int(x)) for x in row) + "\n")
    os.replace(tmp, path)


def front_digest(costs) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(costs, dtype="<u4").tobytes()).hexdigest()[:16]


def _digest_job(args):
    config, seed, d, budget, qi = args
    g, queries = getattr(synth, config)(seed)
    if d:
        g = g.first_objectives(d)
    s, t = queries[qi]
    try:
        f = oracle.solve(g, s, t, label_budget=budget)
    except oracle.OracleError as e:
        if e.code != oracle.BUDGET:
            raise
        return f"{qi} {s} {t} -1 -1 -1 -"
    return (f"{qi} {s} {t} {len(f.costs)} {f.stats['labels']} {f.stats['extracted']} "
            f"{front_digest(f.costs)}")


def shortest_hop_queries(g, queries, k):
    """Indices of the k queries with the fewest hops from start to goal."""
    import numpy as np
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path
    a = sp.csr_matrix((np.ones(len(g.col)), g.col.astype(np.int64), g.rowptr.astype(np.int64)),
                      shape=(g.n, g.n))
    hops = []
    for lo in range(0, len(queries), 32):
        part = queries[lo:lo + 32]
        dist = shortest_path(a, unweighted=True, indices=[s for s, _ in part])
        hops += [int(dist[j, t]) for j, (_, t) in enumerate(part)]
    return sorted(sorted(range(len(queries)), key=lambda i: (hops[i], i))[:k])


def write_digests(args):
    g, queries = getattr(synth, args.config)(args.seed)
    if args.d:
        g = g.first_objectives(args.d)
    sel = shortest_hop_queries(g, queries, args.shortest_hops) if args.shortest_hops else range(len(queries))
    jobs = [(args.config, args.seed, args.d, args.budget, qi) for qi in sel]
    ctx = mp.get_context("spawn")
    found = {}
    with ctx.Pool(args.jobs) as pool:
        for line in pool.imap_unordered(_digest_job, jobs):
            found[int(line.split()[0])] = line
            if len(found) % 64 == 0 or args.shortest_hops:
                print(f"{len(found)}/{len(jobs)} queries", flush=True)
    lines = [found[qi] for qi in sel]
    suffix = f"_d{args.d}" if args.d else ""
    if args.shortest_hops:
        suffix += f"_short{args.shortest_hops}"
    path = os.path.join(HERE, f"{args.config}_seed{args.seed}{suffix}.digests")
    with open(path + ".tmp", "w") as f:
        f.write(f"# oracle fronts (Algorithm 1) as digests; label budget {args.budget or 'none'}"
                + (f"; the {args.shortest_hops} shortest-hop queries" if args.shortest_hops else "") + "\n")
        f.write(f"graph {g.name} {g.digest()}\n")
        f.write("# qi start goal count labels extracted sha256[:16]\n")
        for line in lines:
            f.write(line + "\n")
    os.replace(path + ".tmp", path)
    print(path, len(lines), "queries")


# time-expanded routes with oracle digests: (seed, rows, cols, windows, d)
ROUTES = [(1, 4, 6, 20, 12), (1, 6, 8, 24, 8), (1, 6, 8, 24, 10), (1, 6, 8, 24, 12)]


def _route_job(spec):
    seed, rows, cols, windows, d = spec
    g, q = synth.time_route(seed, rows, cols, windows, d)
    s, t = q[0]
    t0 = time.time()
    f = oracle.solve(g, s, t)
    print(f"{g.name}: {len(f.costs)} solutions, {f.stats['extracted']} extracted, {time.time() - t0:.1f}s",
          flush=True)
    return (f"{g.name} {g.digest()} {s} {t} {len(f.costs)} {f.stats['labels']} {f.stats['extracted']} "
            f"{front_digest(f.costs)}")


def write_routes(args):
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        lines = pool.map(_route_job, ROUTES)
    path = os.path.join(HERE, "routes.digests")
    with open(path + ".tmp", "w") as f:
        f.write("# oracle fronts (Algorithm 1) of time-expanded ship routes (synth.time_route) as digests\n")
        f.write("# name graph-digest start goal count labels extracted sha256[:16]\n")
        for line in lines:
            f.write(line + "\n")
    os.replace(path + ".tmp", path)
    print(path, len(lines), "routes")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config", choices=["config1", "config2", "config3", "config4", "routes"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--queries", default="0:1", help="slice lo:hi of the config's query list")
    ap.add_argument("--d", type=int, default=0, help="use only the first d objectives")
    ap.add_argument("--digests", action="store_true", help="all queries, digest lines")
    ap.add_argument("--jobs", type=int, default=4)
    ap.add_argument("--budget", type=int, default=0, help="oracle label budget per query")
    ap.add_argument("--shortest-hops", type=int, default=0, help="digests of the K fewest-hop queries only")
    args = ap.parse_args()
    if args.config == "routes":
        write_routes(args)
        return
    if args.digests:
        write_digests(args)
        return
    g, queries = getattr(synth, args.config)(args.seed)
    if args.d:
        g = g.first_objectives(args.d)
    lo, hi = (int(x) for x in args.queries.split(":"))
    for qi in range(lo, min(hi, len(queries))):
        s, t = queries[qi]
        t0 = time.time()
        front = oracle.solve(g, s, t)
        dt = time.time() - t0
        suffix = f"_d{args.d}" if args.d else ""
        path = os.path.join(HERE, f"{args.config}_seed{args.seed}{suffix}_q{qi}.front")
        write_front(path, g, s, t, front, note=f"wall {dt:.1f}s")
        print(f"{path}: {len(front.costs)} solutions, {front.stats['labels']} labels, {dt:.1f}s",
              flush=True)


if __name__ == "__main__":
    main()
