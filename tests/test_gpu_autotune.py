"""The lane-plan autotuner (paper_1304_0681_gb300.autotune): it times the
candidate (lanes, rows) plans of every read-length class on a sample of the
caller's batch, installs the fastest with sw_set_plan, and the batch then
aligns exactly as the oracle does (scores, end cells and CIGARs are
integers: zero tolerance)."""
import numpy as np
import pytest

import synth
from gpu_helpers import assert_parity, run_gpu

pytestmark = pytest.mark.gpu
DEFAULT = (5, -4, -10, -1)


@pytest.fixture(autouse=True)
def _reset_plans():
    import paper_1304_0681_gb300 as sw
    sw.sw_set_plan(0, 1, 8)
    yield
    sw.sw_set_plan(0, 1, 8)


def test_candidate_plans_cover_the_class():
    from paper_1304_0681_gb300 import autotune
    import paper_1304_0681_gb300 as sw
    rows = set(sw._swgb.sw_plan_rows())
    for m_max in (16, 75, 100, 150, 250, 400, 800, 2000):
        plans = autotune.candidate_plans(m_max)
        assert plans, m_max
        for lanes, r in plans:
            assert r in rows and 1 <= lanes <= 32
            assert lanes * r >= m_max or lanes == 32


def test_tuned_plans_are_installed_and_exact():
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import autotune
    wl = synth.generate("uneven", seed=31, n_reads=2500)
    lengths = np.unique(wl.read_lengths)
    m, n = wl.pair_read_lengths, wl.window_lengths
    model = {int(L): sw.sw_plan_query(int(L), int(n[m == L].max()), DEFAULT[0]) for L in lengths}
    chosen = autotune.tune(wl, DEFAULT, sample_pairs=600, use_cache=False)
    # one plan per read-length class of the batch (75, 100, 150, 250, 400, 800)
    assert sorted(chosen) == sorted(int(L) for L in lengths)
    for m_max, (lanes, r) in chosen.items():
        assert (lanes, r) in autotune.candidate_plans(m_max) or (lanes, r) == model[m_max]
        # installed: the library's plan for the class is the tuned one
        # wherever the class's score bound allows that many rows (a 16-bit-key
        # class with scores above 510 holds at most 32 rows per lane)
        if r <= 32 or not 510 < DEFAULT[0] * m_max <= 1022:
            assert sw.sw_plan_query(m_max, m_max + 200, DEFAULT[0]) == (lanes, r), m_max
    got = run_gpu(wl, DEFAULT)
    assert_parity(wl, got, DEFAULT)
