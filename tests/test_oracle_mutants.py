"""The oracle's pins catch planted mistakes (CPU only).

Each case copies ``oracle/namoa_oracle.cpp``, plants one plausible mistake by
an exact text replacement, builds the copy with g++ and runs the pins of
``test_oracle.py`` against it through ``oracle.library``. A case passes when
at least one pin rejects the mutant; the unmodified copy must pass them all.
No mistake is planted in the oracle the other tests use.

Mutants that cannot change any result are not listed. Two examples:
- A strict instead of weak test against P. An equal-cost goal label is
  already a Duplicate at the goal's frontier, so P never receives it.
- PruneOPEN with the inequality reversed, as printed in Sec. 3. Labels leave
  OPEN in lexicographic order of F, so every OPEN label l* has F(l*) >= g(l)
  lexicographically. The reversed test F(l*) <= g(l) then only holds when
  F(l*) = g(l), and such labels complete to equal or dominated costs.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from pins import brute_front, check_front, dijkstra, lex_dijkstra

SRC = os.path.join(os.path.dirname(oracle.__file__), "namoa_oracle.cpp")

# name: (text in namoa_oracle.cpp, replacement)
MUTANTS = {
    "arc cost of the wrong objective": (
        "g2[i] = pool.g(l)[i] + G.c(i, e);", "g2[i] = pool.g(l)[i] + G.c(0, e);"),
    "inadmissible heuristic in F": (
        "F2[i] = g2[i] + hv(i, vp);", "F2[i] = g2[i] + 2 * hv(i, vp);"),
    "heuristic of the wrong objective": (
        "uint64_t nd = dv + G.c(k, rarc[i]);", "uint64_t nd = dv + G.c(0, rarc[i]);"),
    "heuristic taken at the arc's source node": (
        "F2[i] = g2[i] + hv(i, vp);", "F2[i] = g2[i] + hv(i, v);"),
    "dominance ignores the last objective": (
        "  bool less = false;\n  for (int i = 0; i < d; ++i) {",
        "  bool less = false;\n  for (int i = 0; i + 1 < d; ++i) {"),
    "path records a wrong arc": (
        "if (S.pool.parent[x] != kNone) edges.push_back(S.pool.edge[x]);",
        "if (S.pool.parent[x] != kNone) edges.push_back(S.pool.edge[x] ^ 1);"),
    "OPEN pops in reverse lexicographic order": (
        "if (A[i] != B[i]) return A[i] < B[i];", "if (A[i] != B[i]) return A[i] > B[i];"),
}


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.cpp"
    src.write_text(text)
    lib = tmp_path / f"{name}.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", str(lib), str(src)])
    return str(lib)


def _tuples(costs):
    return [tuple(int(x) for x in r) for r in costs]


def _pins_hold() -> bool:
    """A compact run of the oracle pins; False on the first one that fails."""
    try:
        for seed in range(24):
            n, d = 5 + seed % 5, 1 + seed % 5
            g = synth.random_digraph(seed, n, d, p=0.35, cmax=3)
            res = oracle.solve(g, 0, n - 1)
            assert _tuples(res.costs) == brute_front(g, 0, n - 1)
            check_front(g, 0, n - 1, res.costs, res.paths)
        for rows, cols, d, seed in [(3, 3, 2, 1), (3, 4, 3, 2), (3, 4, 5, 3), (2, 5, 4, 4)]:
            g = synth.small_grid(seed, rows, cols, d, cmin=0, cmax=4)
            res = oracle.solve(g, 0, g.n - 1)
            assert _tuples(res.costs) == brute_front(g, 0, g.n - 1)
            check_front(g, 0, g.n - 1, res.costs, res.paths)
        g, q = synth.config1()
        s, t = q[0]
        h = oracle.heuristic(g, t)
        for k in range(g.d):
            ref = dijkstra(g, t, k, reverse=True)
            assert all(int(h[k, v]) == ref[v] for v in range(g.n))
        res = oracle.solve(g, s, t)
        for k in range(g.d):
            assert res.costs[:, k].astype(np.int64).min() == dijkstra(g, s, k)[t]
        assert _tuples(res.costs)[0] == lex_dijkstra(g, s, t)
        check_front(g, s, t, res.costs, res.paths)
        assert res.stats["pruned_closed"] == 0 and res.stats["pruned_p"] == 0
        return True
    except (AssertionError, oracle.OracleError):
        return False


def test_unmodified_copy_passes_the_pins(tmp_path):
    lib = _build(tmp_path, "control", open(SRC).read())
    with oracle.library(lib):
        assert _pins_hold()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_the_mutant(tmp_path, name):
    text = open(SRC).read()
    old, new = MUTANTS[name]
    assert text.count(old) == 1, "the mutation site moved"
    lib = _build(tmp_path, "mutant", text.replace(old, new))
    with oracle.library(lib):
        assert not _pins_hold(), f"no pin caught: {name}"
