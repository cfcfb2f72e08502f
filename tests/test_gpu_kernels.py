"""Kernel-level checks: single device routines of a search step, run through
the test hooks of include/opmos_test.h on chosen inputs, against plain host
references of the same operation.

* The merge of one node (Algorithm 1's frontier checks with the in-batch
  resolution of Sec. 5), by one warp, one block, or a block merge split
  over several ranges of the frontier: the frontier afterwards must be the
  Pareto-minimal,
  cost-unique set of the old frontier and the candidates, with an old entry
  kept over an equal candidate and, among equal candidates, the one with the
  smallest arc id. Frontier and candidate counts cross the 32-entry tile, the
  32-candidate batch, the slot count and the 512-entry block-merge threshold.
* The window of the ordered extraction (Algorithm 2): the live entries in
  the histogram bins [0, b*], b* the largest bin whose cumulative count stays
  within W (at least the first non-empty one) -- and, independently of the
  bins, a lexicographic prefix of the live entries (of their F[0] bucket and
  F[1]; with bucket width 1, of F).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def op():
    import paper_2411_16667_gb300 as pkg
    pkg.build()
    from paper_2411_16667_gb300 import opmos
    if opmos.opmos_device_count() == 0:
        pytest.fail("no CUDA device visible to the library")
    return opmos


def _antichain(rng, n, d, hi):
    """Up to n mutually non-dominated, distinct d-vectors: draws on the plane
    sum = hi * d / 2 (equal sums never dominate unless equal), deduplicated."""
    if d == 1:
        return rng.integers(0, hi, size=(min(n, 1), 1)).astype(np.uint32)
    x = rng.integers(0, hi, size=(4 * n + 16, d)).astype(np.int64)
    x[:, -1] = hi * d // 2 - x[:, :-1].sum(axis=1)
    x = x[x[:, -1] >= 0]
    x = np.unique(x, axis=0)
    rng.shuffle(x)
    return x[:n].astype(np.uint32)


def _reference(front, cand, arc):
    """Host merge: Pareto-minimal unique set of front + cand with the tie
    rules; returns sorted [(cost tuple, origin)]."""
    nf = len(front)
    allv = np.concatenate([front.astype(np.int64).reshape(-1, cand.shape[1]), cand.astype(np.int64)])
    # rank for ties: old entries first (by index), then candidates by arc id
    tie = np.concatenate([np.arange(nf), nf + np.argsort(np.argsort(arc, kind="stable"), kind="stable")])
    keep = []
    for i, x in enumerate(allv):
        le = np.all(allv <= x, axis=1)
        lt = np.any(allv < x, axis=1)
        if np.any(le & lt):
            continue
        eq = le & ~lt
        if np.any(eq & (tie < tie[i])):
            continue
        keep.append((tuple(int(v) for v in x), i))
    return sorted(keep)


CASES = [  # (d, frontier size, candidates, slots, overflow lists)
    (1, 1, 5, 32, 1), (2, 31, 20, 32, 32), (2, 32, 33, 32, 1), (3, 33, 31, 32, 8), (3, 100, 70, 32, 32),
    (3, 511, 40, 128, 32), (3, 512, 33, 32, 2), (4, 513, 64, 32, 8), (5, 200, 100, 128, 8), (8, 60, 45, 32, 32),
    (3, 3000, 50, 32, 1), (12, 40, 40, 32, 4), (16, 25, 35, 32, 32), (2, 0, 40, 32, 16),
    # many candidates beyond the slots: several rounds over the lists, groups of a block merge
    (3, 600, 700, 32, 32), (2, 50, 300, 16, 32), (5, 300, 1000, 64, 8), (4, 150, 530, 128, 16), (3, 80, 200, 8, 1),
    # many slot candidates: split merges whose parts split the candidates (and groups of 256 within a part)
    (3, 900, 1000, 1024, 32), (2, 2000, 600, 1024, 32), (4, 300, 700, 512, 8), (8, 200, 400, 1024, 32),
    (3, 5000, 90, 1024, 32)]


@pytest.mark.parametrize("d,nf,nc,slots,lists", CASES)
@pytest.mark.parametrize("block", [0, 1, 3, 8])
def test_node_merge_matches_host_reference(op, d, nf, nc, slots, lists, block):
    """block: 0 one warp, 1 one block, 3 or 8 a block merge split into that
    many parts (ranges of the slot candidates times ranges of the frontier;
    candidates beyond the slots go through the lists after the parts)."""
    rng = np.random.default_rng(1000 * d + nf + nc + int(block))
    hi = 40 if nf < 400 else 400
    front = _antichain(rng, nf, d, hi) if nf else np.zeros((0, d), np.uint32)
    nf = len(front)
    cand = rng.integers(0, hi, size=(nc, d)).astype(np.uint32)
    if nf:  # ties and dominance against the frontier: copies and nudged copies of its entries
        pick = rng.integers(0, nf, size=nc // 3)
        cand[: nc // 3] = front[pick]
        cand[nc // 3: nc // 3 + nc // 6] = front[rng.integers(0, nf, size=nc // 6)] + 1
    cand[-3:] = cand[0]  # equal candidates: the smallest arc must win
    if nf < 40:
        cand[-4] = 0      # the zero vector dominates everything non-zero
    arc = rng.permutation(10 * nc)[:nc].astype(np.uint32)
    costs, origin = op.opmos_test_merge(front, cand, arc, block, slots, lists)
    got = sorted((tuple(int(v) for v in c), int(o)) for c, o in zip(costs, origin))
    assert got == _reference(front, cand, arc)


NB, SUB = 4096, 256


def _bin(f0, f1, b0, b1, s1, delta, s2):
    """The histogram bin a search step assigns to F = (f0, f1): cell
    q * 256 + x with q the F[0] bucket (width delta from b0) and x the F[1]
    cell (F[1] >> s1 from b1, at most 255); 2^s2 cells per bin; the last bin
    collects the rest."""
    q = (f0 - b0) // delta if f0 > b0 else 0
    x = min((f1 - b1) >> s1, SUB - 1) if f1 > b1 else 0
    return min((q * SUB + x) >> s2, NB - 1)


@pytest.mark.parametrize("n,window,spread,s1,delta,s2,seed", [
    (1000, 64, 30, 0, 1, 0, 1), (1000, 256, 30, 2, 1, 1, 2), (5000, 1024, 200, 3, 2, 3, 3),
    (300, 5000, 10, 0, 1, 0, 4), (4000, 100, 3, 0, 1, 0, 5), (20000, 2048, 2000, 6, 4, 5, 6),
    (33, 1, 5, 0, 1, 0, 7), (8000, 700, 60, 4, 1, 8, 8)])
def test_window_is_a_lexicographic_prefix(op, n, window, spread, s1, delta, s2, seed):
    rng = np.random.default_rng(seed)
    f0 = (500 + rng.integers(0, spread, size=n)).astype(np.uint32)
    f1 = (7000 + rng.integers(0, 40 * spread, size=n)).astype(np.uint32)
    dead = rng.random(n) < 0.2
    b0, b1 = int(f0.min()), int(f1.min())
    taken, bstar = op.opmos_test_window(f0, f1, dead, window, [b0, b1, s1, delta, s2])
    live = ~dead
    assert not np.any(taken & dead)
    bins = np.array([_bin(int(a), int(b), b0, b1, s1, delta, s2) for a, b in zip(f0, f1)])
    hist = np.bincount(bins[live], minlength=NB)
    cum = np.cumsum(hist)
    first = int(np.flatnonzero(hist[:NB - 1])[0])
    fit = np.flatnonzero(cum[:NB - 1] <= window)
    exp_bstar = max(int(fit[-1]) if fit.size else 0, first)
    assert bstar == exp_bstar
    assert np.array_equal(taken, live & (bins <= exp_bstar))
    # a lexicographic prefix of the live entries in (F0 bucket, F1) order --
    # (F0, F1) order when delta = 1 -- whatever the bins
    q = (f0.astype(np.uint64) - np.uint64(b0)) // np.uint64(delta)
    keys = (q << np.uint64(32)) | f1.astype(np.uint64)
    if taken.any() and (live & ~taken).any():
        assert keys[taken].max() < keys[live & ~taken].min()
    assert taken.sum() <= window or np.all(bins[taken] == first)
