"""CUDA graphs: sw_batch_align itself and plans (sw_plan_*) enqueue a fixed
sequence of launches with no host wait, so a captured call replays with the
oracle's results bit for bit -- also after the batch's bases change under a
fixed shape; a plan reports a changed shape instead of running it, and a
call that would have to allocate during a capture is refused."""
import numpy as np
import pytest

import synth
from gpu_helpers import assert_parity

pytestmark = pytest.mark.gpu
DEFAULT = (5, -4, -10, -1)


def _batch(wl):
    from paper_1304_0681_gb300 import DeviceBatch
    return DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets,
                                   cigar=True)


def _outputs(b):
    end = b.end.cpu().numpy().reshape(-1, 2)
    return {"score": b.score.cpu().numpy().astype(np.int64), "i_end": end[:, 0].astype(np.int64),
            "j_end": end[:, 1].astype(np.int64), "ops": b.cigar_ops.cpu().numpy().view(np.uint32),
            "cigar_offsets": b.cigar_offsets.cpu().numpy(), "n_ops": b.cigar_n.cpu().numpy().astype(np.int64)}


def _clear(b):
    b.score.fill_(-7)
    b.end.fill_(-7)
    b.cigar_n.fill_(-7)


def _same_shape_new_bases(wl, seed):
    rng = np.random.default_rng(seed)
    reads = rng.integers(0, 4, len(wl.reads)).astype(np.uint8)
    wins = wl.windows.copy()
    # keep a planted copy of each read in its window where it fits, so the
    # new batch still has long alignments
    for p in range(wl.n_pairs):
        r0, r1 = wl.read_offsets[p], wl.read_offsets[p + 1]
        w0, w1 = wl.window_offsets[p], wl.window_offsets[p + 1]
        if (w1 - w0) >= (r1 - r0) + 10:
            wins[w0 + 5:w0 + 5 + (r1 - r0)] = reads[r0:r1]
    return synth.Workload(wl.name + "[new bases]", reads, wl.read_offsets, wins, wl.window_offsets, wl.pair_read,
                          wl.cand_offsets, wl.kinds, wl.true_cand)


def test_plan_execution_matches_oracle():
    from paper_1304_0681_gb300 import BatchPlan
    wl = synth.generate("parity", seed=4)
    b = _batch(wl)
    plan = BatchPlan(b, DEFAULT)
    _clear(b)
    plan.align()
    plan.status()
    assert_parity(wl, _outputs(b), DEFAULT)
    plan.close()


def test_graph_replay_matches_oracle_and_follows_new_bases():
    import torch

    import synth as sy
    from paper_1304_0681_gb300 import BatchPlan
    # several length classes, long reads and spliced windows: every kind of
    # launch the plan makes
    wl = sy.generate("uneven", seed=5, n_reads=600)
    b = _batch(wl)
    plan = BatchPlan(b, DEFAULT)
    plan.align()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=side):
        plan.align()
    _clear(b)
    graph.replay()
    torch.cuda.synchronize()
    plan.status()
    assert_parity(wl, _outputs(b), DEFAULT)
    # same shape, new bases: the captured graph reads the bases at replay
    wl2 = _same_shape_new_bases(wl, 9)
    b.reads.copy_(torch.from_numpy(wl2.packed_reads()).cuda())
    b.windows.copy_(torch.from_numpy(wl2.packed_windows()).cuda())
    _clear(b)
    graph.replay()
    torch.cuda.synchronize()
    plan.status()
    assert_parity(wl2, _outputs(b), DEFAULT)
    del graph
    plan.close()


def test_changed_shape_is_reported():
    import torch

    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import BatchPlan
    wl = synth.generate("parity", seed=6, n_reads=300)
    b = _batch(wl)
    plan = BatchPlan(b, DEFAULT)
    plan.align()
    plan.status()
    # move bases from read 1 to read 0: same total, another read-length class
    ro = b.read_offsets.cpu().numpy().copy()
    ro[1] = ro[0] + 1
    b.read_offsets.copy_(torch.from_numpy(ro).cuda())
    plan.align()
    with pytest.raises(sw.SwError) as e:
        plan.status()
    assert e.value.code == -6  # SW_ERR_DEVICE_INPUT
    plan.close()


def test_plan_arguments_are_checked():
    import paper_1304_0681_gb300 as sw
    wl = synth.generate("parity", seed=7, n_reads=50)
    b = _batch(wl)
    with pytest.raises(sw.SwError):
        sw._swgb.sw_plan_create(b.read_offsets, b.n_reads, b.window_offsets, None, 0, DEFAULT)
    with pytest.raises(sw.SwError):
        sw._swgb.sw_plan_create(b.read_offsets, b.n_reads, b.window_offsets, None, b.n_pairs, (5, 1, -10, -1))
    plan = sw.BatchPlan(b, DEFAULT, cigar=False)
    with pytest.raises(sw.SwError):  # a score-only plan cannot write a CIGAR
        sw._swgb.sw_plan_align(plan.handle, b.reads, b.windows, b.score, b.end, b.cigar_tuple())
    plan.close()


def test_sw_batch_align_itself_is_captured_and_replayed():
    """The default entry point enqueues a fixed sequence of launches with no
    host wait, so sw_batch_align itself is captured in a CUDA graph (after
    one uncaptured call on the capturing stream has set up its scratch) and
    replayed: bit-exact against the oracle, twice, and after new bases of the
    same shape are written into the captured input buffers."""
    import torch

    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import align
    wl = synth.generate("uneven", seed=12, n_reads=700)
    b = _batch(wl)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        align(b, DEFAULT, stream=side)  # the stream's scratch, outside the capture
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        align(b, DEFAULT, stream=side, sync=False)
    for _ in range(2):
        _clear(b)
        graph.replay()
        torch.cuda.synchronize()
        sw.sw_sync_status(side)
        assert_parity(wl, _outputs(b), DEFAULT)
    wl2 = _same_shape_new_bases(wl, 13)
    b.reads.copy_(torch.from_numpy(wl2.packed_reads()).cuda())
    b.windows.copy_(torch.from_numpy(wl2.packed_windows()).cuda())
    _clear(b)
    graph.replay()
    torch.cuda.synchronize()
    sw.sw_sync_status(side)
    assert_parity(wl2, _outputs(b), DEFAULT)
    del graph


def test_capture_that_would_allocate_is_refused():
    """A call whose scratch would have to grow during a capture returns
    SW_ERR_UNSUPPORTED before enqueuing anything, instead of allocating: here
    the stream's only earlier call asked for no CIGAR, so it holds no
    traceback scratch."""
    import torch

    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import align
    wl = synth.generate("parity", seed=14, n_reads=200)
    b = _batch(wl)
    fresh = torch.cuda.Stream()
    fresh.wait_stream(torch.cuda.current_stream())
    align(b, DEFAULT, cigar=False, stream=fresh)
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(graph, stream=fresh):
        try:
            align(b, DEFAULT, cigar=True, stream=fresh, sync=False)
        except sw.SwError as e:
            err = e
    assert err is not None and err.code == -5  # SW_ERR_UNSUPPORTED
    del graph
    # outside a capture the same call allocates and runs
    align(b, DEFAULT, cigar=True, stream=fresh)
    assert_parity(wl, _outputs(b), DEFAULT)
