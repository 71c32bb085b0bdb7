"""Host-side bookkeeping of the learned filter: the choice of (k, tau) for a
best-hit recall target (filter.calibrate) against a brute force that runs
the filter oracle's selection and best hit for every grid point."""
import numpy as np
import pytest

from oracle import filter_oracle as fo


def _brute(pred, score, off, target, ks, taus):
    true_best = fo.best_per_read(score, off)
    best = None
    for k in ks:
        for tau in taus:
            sel = fo.select_candidates(pred, off, k, tau)
            got = fo.best_per_read(score, off, sel)
            recall = float(np.mean(got == true_best))
            aligned = int(sel.sum())
            if recall >= target and (best is None or aligned < best[2]):
                best = (k, float(tau), aligned, recall)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_calibrate_matches_brute_force(seed):
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(seed)
    counts = rng.integers(1, 20, 400)
    off = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    n = int(off[-1])
    score = rng.integers(0, 6, n)                       # many tied scores
    # predictions that track the score, with noise and exact ties
    pred = (score / 6.0 + rng.normal(0, 0.15, n)).astype(np.float32)
    pred[rng.random(n) < 0.1] = 0.5
    ks, taus = (1, 2, 3, 4, 6, 8), [0.0, 0.005, 0.01, 0.02, 0.03, 0.05, 0.08, 0.12, 0.2]
    for target in (0.8, 0.9, 0.97, 1.0):
        got = flt.calibrate(pred, score, off, target, ks=ks, taus=taus)
        want = _brute(pred, score, off, target, ks, taus)
        assert got == want, (target, got, want)


def test_calibrate_reports_none_when_unreachable():
    from paper_1304_0681_gb300 import filter as flt
    off = np.array([0, 3])
    # the best candidate is predicted worst and every margin is wide: with
    # three candidates, k = 1 and k = 2 select without it at either tau
    pred = np.array([0.9, 0.5, 0.0], np.float32)
    score = np.array([1, 2, 9])
    assert flt.calibrate(pred, score, off, 1.0, ks=(1, 2), taus=[0.0, 0.1]) is None
