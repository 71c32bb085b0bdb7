"""Multi-rank sharding on the CPU: world_size 2 over gloo.

Each rank takes its cell-balanced share of the reads (with all of their
candidates), aligns it with the oracle, and the pieces gathered on rank 0
must equal the unsharded run pair for pair and read for read.  The run
counters reduce to the summed units and the slowest rank's time, which is
how the benchmark forms its whole-job value.
"""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1304_0681_gb300.shard import cell_balanced_bounds, read_costs, reduce_run

SCORING = (5, -4, -10, -1)


def test_read_costs_and_bounds_properties():
    wl = synth.generate("filter", seed=11, n_reads=300)
    cost = read_costs(wl.read_lengths, wl.cand_offsets, wl.window_lengths)
    assert int(cost.sum()) == wl.cells()
    for W in (1, 2, 3, 7, 16):
        b = cell_balanced_bounds(wl.read_lengths, wl.cand_offsets, wl.window_lengths, W)
        assert b[0] == 0 and b[-1] == wl.n_reads and np.all(np.diff(b) >= 0)
        shares = np.array([cost[b[k]:b[k + 1]].sum() for k in range(W)])
        assert shares.sum() == cost.sum()
        assert np.all(np.abs(shares - cost.sum() / W) <= 2 * cost.max()), (W, shares)


def test_bounds_edge_cases():
    # fewer reads than ranks: every read lands on exactly one rank
    b = cell_balanced_bounds([100, 100], [0, 1, 2], [200, 200], 5)
    assert b[0] == 0 and b[-1] == 2 and np.all(np.diff(b) >= 0)
    # empty batch
    b = cell_balanced_bounds(np.zeros(0, np.int64), [0], np.zeros(0, np.int64), 3)
    assert list(b) == [0, 0, 0, 0]
    # reads with no candidates or zero length cost nothing
    b = cell_balanced_bounds([0, 50, 50, 0], [0, 0, 2, 3, 3], [10, 10, 10], 2)
    assert list(b) in ([0, 2, 4], [0, 1, 4], [0, 3, 4])
    with pytest.raises(ValueError):
        cell_balanced_bounds([1], [0, 1], [1], 0)


def test_reduce_run_without_process_group():
    assert reduce_run(5, 0.25) == (5.0, 0.25)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = synth.generate("filter", seed=21, n_reads=24)
        b = cell_balanced_bounds(wl.read_lengths, wl.cand_offsets, wl.window_lengths, world)
        part = wl.read_slice(int(b[rank]), int(b[rank + 1]))
        res = oracle.align_batch(part.reads, part.read_offsets, part.windows, part.window_offsets,
                                 pair_read=part.pair_read, scoring=oracle.Scoring(*SCORING), cigar=True, threads=1)
        cig = [oracle.cigar_string(res["ops"][res["cigar_offsets"][p]:res["cigar_offsets"][p] + res["n_ops"][p]])
               for p in range(part.n_pairs)]
        mine = {"rank": rank, "lo": int(b[rank]), "score": res["score"].tolist(), "i_end": res["i_end"].tolist(),
                "j_end": res["j_end"].tolist(), "cigar": cig}
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        units, secs = reduce_run(part.cells(), 0.5 + rank, None)
        if rank == 0:
            import json
            with open(os.path.join(out_dir, "result.json"), "w") as f:
                json.dump({"parts": gathered, "units": units, "secs": secs}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_match_unsharded(tmp_path):
    import json

    import torch.multiprocessing as mp

    import oracle
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    out = json.load(open(tmp_path / "result.json"))
    wl = synth.generate("filter", seed=21, n_reads=24)
    full = oracle.align_batch(wl.reads, wl.read_offsets, wl.windows, wl.window_offsets, pair_read=wl.pair_read,
                              scoring=oracle.Scoring(*SCORING), cigar=True, threads=1)
    parts = sorted(out["parts"], key=lambda d: d["rank"])
    assert parts[0]["lo"] == 0 and parts[1]["lo"] > 0  # both ranks got work
    score = np.concatenate([p["score"] for p in parts])
    np.testing.assert_array_equal(score, full["score"])
    np.testing.assert_array_equal(np.concatenate([p["i_end"] for p in parts]), full["i_end"])
    np.testing.assert_array_equal(np.concatenate([p["j_end"] for p in parts]), full["j_end"])
    cig = sum((p["cigar"] for p in parts), [])
    ref = [oracle.cigar_string(full["ops"][full["cigar_offsets"][p]:full["cigar_offsets"][p] + full["n_ops"][p]])
           for p in range(wl.n_pairs)]
    assert cig == ref
    assert out["units"] == wl.cells()
    assert out["secs"] == 1.5


def _grad_worker(rank, world, port, out_dir):
    """Each rank takes its share of one minibatch, computes the mean
    gradient of its share (the fp64 oracle stands in for the GPU kernel on
    this CPU test) and combines it with the filter's all-reduce."""
    import torch
    import torch.distributed as dist

    from oracle import filter_oracle as fo
    from paper_1304_0681_gb300.filter import allreduce_mean_gradient, minibatch_share
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)
        X = rng.random((37, fo.N_FEAT))
        t = rng.random(37)
        P = fo.Params.init(3)
        lo, hi = minibatch_share(len(t), rank, world)
        g = torch.from_numpy(fo.backward(P, X[lo:hi], t[lo:hi]) if hi > lo else np.zeros(fo.N_PARAMS))
        allreduce_mean_gradient(g, hi - lo, len(t))
        if rank == 0:
            np.save(os.path.join(out_dir, "grad.npy"), g.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_filter_gradient_allreduce_equals_one_rank(tmp_path, world):
    import torch.multiprocessing as mp

    from oracle import filter_oracle as fo
    from paper_1304_0681_gb300.filter import minibatch_share
    mp.spawn(_grad_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    rng = np.random.default_rng(5)
    X = rng.random((37, fo.N_FEAT))
    t = rng.random(37)
    want = fo.backward(fo.Params.init(3), X, t)
    np.testing.assert_allclose(np.load(tmp_path / "grad.npy"), want, rtol=1e-12, atol=1e-14)
    shares = [minibatch_share(37, r, world) for r in range(world)]
    assert shares[0][0] == 0 and shares[-1][1] == 37
    assert all(a[1] == b[0] for a, b in zip(shares, shares[1:]))
