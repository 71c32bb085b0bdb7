"""Host-side bookkeeping of the learned filter: the choice of (k, tau,
delta) for a best-hit recall target (filter.calibrate, and per read-length
class filter.calibrate_by_length) against brute forces that run the filter
oracle's selection and best hit for every grid point."""
import itertools

import numpy as np
import pytest

from oracle import filter_oracle as fo


def _brute(pred, score, off, target, ks, taus, deltas):
    true_best = fo.best_per_read(score, off)
    best = None
    for k in ks:
        for delta in deltas:
            for tau in taus:
                sel = fo.select_candidates(pred, off, k, tau, delta)
                got = fo.best_per_read(score, off, sel)
                recall = float(np.mean(got == true_best))
                aligned = int(sel.sum())
                if recall >= target and (best is None or aligned < best[3]):
                    best = (k, float(tau), float(delta), aligned, recall)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_calibrate_matches_brute_force(seed):
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 20, 400)                   # reads without candidates too
    off = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    n = int(off[-1])
    score = rng.integers(0, 6, n)                       # many tied scores
    # predictions that track the score, with noise and exact ties
    pred = (score / 6.0 + rng.normal(0, 0.15, n)).astype(np.float32)
    pred[rng.random(n) < 0.1] = 0.5
    ks, taus, deltas = (1, 2, 3, 5, 8), [0.0, 0.01, 0.03, 0.08, 0.2], [0.0, 0.05, 0.125, 0.3]
    for target in (0.8, 0.9, 0.97, 1.0):
        got = flt.calibrate(pred, score, off, target, ks=ks, taus=taus, deltas=deltas)
        want = _brute(pred, score, off, target, ks, taus, deltas)
        assert got == want, (target, got, want)


def test_calibrate_reports_none_when_unreachable():
    from paper_1304_0681_gb300 import filter as flt
    off = np.array([0, 3])
    # the best candidate is predicted worst and every margin is wide: with
    # three candidates, k = 1 and k = 2 select without it at either tau
    pred = np.array([0.9, 0.5, 0.0], np.float32)
    score = np.array([1, 2, 9])
    assert flt.calibrate(pred, score, off, 1.0, ks=(1, 2), taus=[0.0, 0.1], deltas=[0.0, 0.3]) is None
    # a delta that reaches the best candidate's prediction makes it reachable
    assert flt.calibrate(pred, score, off, 1.0, ks=(1,), taus=[0.0], deltas=[0.0, 1.0])[:3] == (1, 0.0, 1.0)


@pytest.mark.parametrize("top,times", [(1, 4), (2, 3), (1, 1)])
def test_oversample_top_against_a_loop(top, times):
    """The training multiset of filter.oversample_top: every row once, plus
    each read's `top` best rows (score descending, lower index first on
    ties) `times - 1` more times; checked against a per-read loop."""
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(top * 10 + times)
    counts = rng.integers(0, 9, 300)
    off = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    score = rng.integers(0, 4, int(off[-1]))            # ties on purpose
    got = np.sort(flt.oversample_top(score, off, top, times))
    want = list(range(int(off[-1])))
    for r in range(len(counts)):
        rows = sorted(range(off[r], off[r + 1]), key=lambda p: (-score[p], p))
        for p in rows[:top]:
            want += [p] * (times - 1)
    np.testing.assert_array_equal(got, np.sort(np.array(want, dtype=np.int64)))


@pytest.mark.parametrize("seed", range(4))
def test_calibrate_by_length_matches_brute_force(seed):
    """filter.calibrate_by_length reaches the fewest aligned cells of any
    per-class choice on its grid (a brute force over every combination, from
    per-class outcomes that the filter oracle's selection computes), and its
    rules, run through the oracle's select_by_length, give the cells and
    recall it reports."""
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(100 + seed)
    nr = 240
    read_len = rng.choice([50, 100, 300], nr)           # length classes <= 80, <= 112, <= 320
    counts = rng.integers(0, 12, nr)
    off = np.zeros(nr + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    n = int(off[-1])
    win_len = rng.integers(100, 400, n)
    score = rng.integers(0, 6, n)
    noise = np.where(np.repeat(read_len, counts) > 100, 0.08, 0.25)   # long reads rank better
    pred = (score / 6.0 + rng.normal(0, 1, n) * noise).astype(np.float32)
    pred[rng.random(n) < 0.05] = 0.5
    ks, taus, deltas = (1, 2, 4), [0.0, 0.05], [0.0, 0.1]
    grid = [(k, t, d) for k in ks for d in deltas for t in taus]
    true_best = fo.best_per_read(score, off)
    cells_of = np.repeat(read_len, counts) * win_len
    per = {}
    for L in (50, 100, 300):
        rows = []
        for k, t, d in grid:
            sel = fo.select_candidates(pred, off, k, t, d)
            got = fo.best_per_read(score, off, sel)
            in_cls = read_len == L
            miss = int(np.sum((got != true_best) & in_cls))
            cells = int(cells_of[sel & np.repeat(in_cls, counts)].sum())
            rows.append((miss, cells))
        per[L] = rows
    for target in (0.85, 0.95, 1.0):
        need = int(np.ceil(target * nr - 1e-9))
        want = None
        for combo in itertools.product(range(len(grid)), repeat=3):
            miss = sum(per[L][i][0] for L, i in zip((50, 100, 300), combo))
            cells = sum(per[L][i][1] for L, i in zip((50, 100, 300), combo))
            if nr - miss >= need and (want is None or cells < want):
                want = cells
        got = flt.calibrate_by_length(pred, score, off, read_len, win_len, target, ks=ks, taus=taus, deltas=deltas)
        if want is None:
            assert got is None
            continue
        rules, cells, pairs, recall = got
        assert cells == want, (target, cells, want)
        sel = fo.select_by_length(pred, off, read_len, rules)
        assert int(cells_of[sel].sum()) == cells and int(sel.sum()) == pairs
        assert float(np.mean(fo.best_per_read(score, off, sel) == true_best)) == recall >= need / nr
