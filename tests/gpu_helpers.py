"""Helpers for the GPU parity tests: run a workload through the C ABI and
compare it with the oracle element by element."""
from __future__ import annotations

import numpy as np

import oracle


def run_gpu(wl, scoring, cigar: bool = True, indexed: bool | None = None, stream=None):
    """Align a synth.Workload on the GPU; returns numpy score, i_end, j_end
    and the CSR CIGAR."""
    import torch
    from paper_1304_0681_gb300 import DeviceBatch, align

    if indexed is None:
        indexed = not np.array_equal(wl.pair_read, np.arange(wl.n_pairs))
    if indexed:
        b = DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets,
                                    pair_read=wl.pair_read, cigar=cigar)
    else:
        b = DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets,
                                    cigar=cigar)
    align(b, scoring, cigar=cigar, stream=stream)
    torch.cuda.synchronize()
    end = b.end.cpu().numpy().reshape(-1, 2)
    out = {"score": b.score.cpu().numpy().astype(np.int64), "i_end": end[:, 0].astype(np.int64),
           "j_end": end[:, 1].astype(np.int64)}
    if cigar:
        out["ops"] = b.cigar_ops.cpu().numpy().view(np.uint32)
        out["cigar_offsets"] = b.cigar_offsets.cpu().numpy()
        out["n_ops"] = b.cigar_n.cpu().numpy().astype(np.int64)
    return out


def oracle_subset(wl, pairs, scoring, cigar=True):
    sub = wl.pair_slice(pairs)
    return oracle.align_batch(sub.reads, sub.read_offsets, sub.windows, sub.window_offsets,
                              scoring=oracle.Scoring(*scoring), cigar=cigar)


def assert_parity(wl, got, scoring, pairs=None, cigar=True):
    """Bit-exact score, end and CIGAR of the given pairs (all by default)."""
    pairs = np.arange(wl.n_pairs) if pairs is None else np.asarray(pairs)
    ref = oracle_subset(wl, pairs, scoring, cigar)
    bad = []
    for k, p in enumerate(pairs):
        g = (got["score"][p], got["i_end"][p], got["j_end"][p])
        r = (ref["score"][k], ref["i_end"][k], ref["j_end"][k])
        if g != r:
            bad.append((int(p), "end/score", g, r))
            continue
        if cigar:
            go = got["cigar_offsets"][p]
            gops = got["ops"][go:go + got["n_ops"][p]]
            ro = ref["cigar_offsets"][k]
            rops = ref["ops"][ro:ro + ref["n_ops"][k]]
            if not np.array_equal(gops, rops):
                bad.append((int(p), "cigar", oracle.cigar_string(gops), oracle.cigar_string(rops)))
    assert not bad, f"{len(bad)} of {len(pairs)} pairs differ; first: {bad[:5]}"
