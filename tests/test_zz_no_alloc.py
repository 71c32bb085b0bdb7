"""sw_batch_align_noalloc: the entry point for callers that cannot let the
library allocate device memory (their memory belongs to their own pool, or
cudaMalloc's device synchronisation is unacceptable to them).  It keeps its
scratch in a fixed static device array, so the test checks that two calls in
a row -- the second one inheriting the first one's leftover scratch contents
-- each give exactly what sw_batch_align gives for the same batch, and what
the CPU oracle gives (scores and end cells are integers: the tolerance is
zero), and that sizes beyond the array's limits are refused with a clear
error.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SCORING = (5, -4, -10, -1)


def _batch(wl):
    from paper_1304_0681_gb300 import DeviceBatch
    return DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets,
                                   cigar=False)


def _reference(wl):
    import torch
    from paper_1304_0681_gb300 import align
    b = _batch(wl)
    align(b, SCORING, cigar=False)
    torch.cuda.synchronize()
    return b.score.cpu().numpy(), b.end.cpu().numpy()


def _noalloc(wl):
    import torch
    import paper_1304_0681_gb300 as sw
    b = _batch(wl)
    b.score.fill_(-7)
    b.end.fill_(-7)
    sw.sw_batch_align_noalloc(b.reads, b.read_offsets, b.windows, b.window_offsets, b.n_pairs, SCORING,
                              b.score, b.end)
    torch.cuda.synchronize()
    return b.score.cpu().numpy(), b.end.cpu().numpy()


def _mixed(seed, n):
    """Reads of 1..1024 bases, windows of 0..1100 (some empty), and true
    matches planted in about a third of the pairs."""
    wl = synth.random_pairs(n, (1, 1024), (0, 1100), seed=seed)
    rng = np.random.default_rng(seed)
    for p in rng.choice(n, n // 3, replace=False):
        r0, r1 = wl.read_offsets[p], wl.read_offsets[p + 1]
        w0, w1 = wl.window_offsets[p], wl.window_offsets[p + 1]
        L = min(r1 - r0, w1 - w0)
        wl.windows[w0:w0 + L] = wl.reads[r0:r0 + L]
    return wl


def _oracle(wl):
    o = oracle.align_batch(wl.reads, wl.read_offsets, wl.windows, wl.window_offsets,
                           scoring=oracle.Scoring(*SCORING), cigar=False)
    return o["score"], np.stack([o["i_end"], o["j_end"]], axis=1).ravel()


def test_two_calls_match_sw_batch_align_and_the_oracle():
    first = _mixed(1, 3000)
    second = synth.generate("parity", seed=9, n_reads=700)  # smaller batch after a larger one
    for wl in (first, second):
        ref_s, ref_e = _reference(wl)
        got_s, got_e = _noalloc(wl)
        np.testing.assert_array_equal(got_s, ref_s)
        np.testing.assert_array_equal(got_e, ref_e)
        orc_s, orc_e = _oracle(wl)
        np.testing.assert_array_equal(got_s, orc_s)
        np.testing.assert_array_equal(got_e, orc_e)
    assert (ref_s > 0).all()


def test_limits_are_refused():
    import paper_1304_0681_gb300 as sw
    wl = synth.generate("parity", seed=4, n_reads=8)
    b = _batch(wl)
    with pytest.raises(sw.SwError) as ei:   # more pairs than the static array holds
        sw.sw_batch_align_noalloc(b.reads, b.read_offsets, b.windows, b.window_offsets,
                                  262145, SCORING, b.score, b.end)
    assert ei.value.code == -5
    long_read = synth.random_pairs(4, (1025, 1100), (50, 60), seed=5)
    b2 = _batch(long_read)
    with pytest.raises(sw.SwError) as ei:   # a read longer than 1024 bases
        sw.sw_batch_align_noalloc(b2.reads, b2.read_offsets, b2.windows, b2.window_offsets, b2.n_pairs,
                                  SCORING, b2.score, b2.end)
    assert ei.value.code == -5
    # still usable afterwards
    ref_s, ref_e = _reference(wl)
    got_s, got_e = _noalloc(wl)
    np.testing.assert_array_equal(got_s, ref_s)
    np.testing.assert_array_equal(got_e, ref_e)
