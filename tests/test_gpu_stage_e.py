"""GPU parity of Stage E task iv (records, splice junctions) against
oracle/stage_e_oracle.py.  The oracle side runs on the oracle's own
alignments; the GPU side on the GPU's.  Records and junction counts are
integers: compared exactly (junctions as a set, since the table's order is
its slot order)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import stage_e_oracle as se

pytestmark = pytest.mark.gpu
DEFAULT = (5, -4, -10, -1)


def _planted(n, seed):
    """Reads of 100 bases over {A,C,G} split by an intron of random length
    with GT-AG, CT-AC or other marks, in T flanks; plus random pairs."""
    rng = np.random.default_rng(seed)
    enc = {c: i for i, c in enumerate("ACGT")}
    marks = [("GT", "AG"), ("CT", "AC"), ("AA", "TT"), ("GT", "AC")]
    reads, wins = [], []
    for k in range(n):
        if k % 5 == 4:
            reads.append(rng.integers(0, 4, rng.integers(20, 120)).astype(np.uint8))
            wins.append(rng.integers(0, 4, rng.integers(50, 300)).astype(np.uint8))
            continue
        mk = marks[rng.integers(0, len(marks))]
        r = rng.choice(list("ACG"), 100)
        r[49] = next(b for b in "ACG" if b != mk[1][1])
        r[50] = next(b for b in "ACG" if b != mk[0][0])
        r = "".join(r)
        L = int(rng.integers(10, 300))
        w = "T" * int(rng.integers(5, 40)) + r[:50] + mk[0] + "T" * (L - 4) + mk[1] + r[50:] + "T" * 20
        reads.append(np.array([enc[c] for c in r], np.uint8))
        wins.append(np.array([enc[c] for c in w], np.uint8))
    roff = np.zeros(n + 1, np.int64)
    np.cumsum([len(x) for x in reads], out=roff[1:])
    woff = np.zeros(n + 1, np.int64)
    np.cumsum([len(x) for x in wins], out=woff[1:])
    return synth.Workload("planted", np.concatenate(reads), roff, np.concatenate(wins), woff,
                          np.arange(n, dtype=np.int64), np.arange(n + 1, dtype=np.int64), np.zeros(n, np.uint8),
                          np.zeros(n, np.int32))


def _coords(wl, seed):
    rng = np.random.default_rng(seed)
    chrom = (np.arange(wl.n_pairs) % 5).astype(np.int32)
    pos = (wl.window_offsets[:-1] + rng.integers(0, 1000, wl.n_pairs)).astype(np.int64)
    strand = (np.arange(wl.n_pairs) % 2).astype(np.int8)
    return chrom, pos, strand


def _gpu_batch(wl):
    import torch
    from paper_1304_0681_gb300 import DeviceBatch, align
    b = DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets,
                                cigar=True)
    align(b, DEFAULT, cigar=True)
    torch.cuda.synchronize()
    return b


def _oracle_side(wl, chrom, pos, strand, min_score, min_intron):
    res = oracle.align_batch(wl.reads, wl.read_offsets, wl.windows, wl.window_offsets,
                             scoring=oracle.Scoring(*DEFAULT), cigar=True)
    cig = se.cigars_of(res)
    recs = se.records(res["score"], res["i_end"], res["j_end"], cig, chrom, pos, strand, min_score)
    jn = se.junction_counts(wl.windows, wl.window_offsets, res["score"], res["j_end"], cig, chrom, pos, min_score,
                            min_intron)
    return recs, jn


def _check(wl, min_score, min_intron, seed):
    import torch

    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import stage_e
    chrom, pos, strand = _coords(wl, seed)
    b = _gpu_batch(wl)
    dc, dp, ds = (torch.from_numpy(x).cuda() for x in (chrom, pos, strand))
    got = stage_e.records(b, dc, dp, ds, min_score)
    sw.sw_sync_status()
    tab = stage_e.JunctionTable(1 << 14)
    tab.detect(b, dc, dp, min_score, min_intron)
    sw.sw_sync_status()
    jn = tab.export()
    recs, jref = _oracle_side(wl, chrom, pos, strand, min_score, min_intron)
    ref = np.array(recs, dtype=np.int64).reshape(-1, 8)
    np.testing.assert_array_equal(got["pair"], ref[:, 0])
    np.testing.assert_array_equal(got["score"], ref[:, 1])
    np.testing.assert_array_equal(got["chrom"], ref[:, 2])
    np.testing.assert_array_equal(got["ref_start"], ref[:, 3])
    np.testing.assert_array_equal(got["ref_end"], ref[:, 4])
    np.testing.assert_array_equal(got["read_start"], ref[:, 5])
    np.testing.assert_array_equal(got["read_end"], ref[:, 6])
    np.testing.assert_array_equal(got["strand"], ref[:, 7])
    gj = {(int(c), int(s), int(e), int(t)): int(n)
          for c, s, e, t, n in zip(jn["chrom"], jn["start"], jn["end"], jn["strand"], jn["count"])}
    assert gj == jref
    return b, tab, (dc, dp), jref


def test_planted_introns():
    wl = _planted(400, seed=1)
    b, tab, coords, jref = _check(wl, min_score=200, min_intron=10, seed=2)
    assert len(jref) > 100 and {k[3] for k in jref} == {0, 1}


@pytest.mark.parametrize("mode", ["tb_auto", "tb_int32"])
def test_uneven_sample(mode):
    import paper_1304_0681_gb300 as sw
    sw.sw_set_traceback_mode(sw.SW_TB_INT32 if mode == "tb_int32" else sw.SW_TB_AUTO)
    try:
        wl = synth.generate("uneven", seed=11, n_reads=700)
        _check(wl, min_score=150, min_intron=20, seed=3)
    finally:
        sw.sw_set_traceback_mode(sw.SW_TB_AUTO)


def test_counts_accumulate_and_clear():
    import paper_1304_0681_gb300 as sw
    wl = _planted(100, seed=4)
    b, tab, (dc, dp), jref = _check(wl, min_score=200, min_intron=10, seed=5)
    tab.detect(b, dc, dp, 200, 10)
    sw.sw_sync_status()
    jn = tab.export()
    got = {(int(c), int(s), int(e), int(t)): int(n)
           for c, s, e, t, n in zip(jn["chrom"], jn["start"], jn["end"], jn["strand"], jn["count"])}
    assert got == {k: 2 * v for k, v in jref.items()}
    tab.clear()
    assert len(tab.export()["count"]) == 0


def test_full_table_and_unsupported_keys_are_reported():
    import torch

    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import stage_e
    wl = _planted(400, seed=6)
    b = _gpu_batch(wl)
    chrom, pos, strand = _coords(wl, 7)
    dc, dp = torch.from_numpy(chrom).cuda(), torch.from_numpy(pos).cuda()
    small = stage_e.JunctionTable(64)  # fewer slots than junctions
    small.detect(b, dc, dp, 200, 10)
    with pytest.raises(sw.SwError) as e:
        sw.sw_sync_status()
    assert e.value.code == -2  # SW_ERR_CAPACITY
    assert len(small.export()["count"]) == 64
    big = stage_e.JunctionTable(1 << 12)
    big.detect(b, torch.full_like(dc, 5000), dp, 200, 10)
    with pytest.raises(sw.SwError) as e:
        sw.sw_sync_status()
    assert e.value.code == -5  # SW_ERR_UNSUPPORTED
    with pytest.raises(sw.SwError):
        stage_e.JunctionTable(100)  # not a power of two


def _top_hits_gpu(score, off, mask, outputs=True):
    import torch
    from paper_1304_0681_gb300 import _swgb
    n = len(off) - 1
    s = torch.from_numpy(np.asarray(score, np.int32)).cuda()
    o = torch.from_numpy(np.asarray(off, np.int64)).cuda()
    m = None if mask is None else torch.from_numpy(np.asarray(mask, np.uint8)).cuda()
    out = [torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda") for _ in range(4)]
    _swgb.sw_top_hits(s, o, n, m, out[0], out[1] if outputs else None, out[2] if outputs else None,
                      out[3] if outputs else None)
    torch.cuda.synchronize()
    return [x[:n].cpu().numpy() for x in out]


def test_top_hits_random_scores():
    """Seeded scores over a narrow range (ties everywhere), 0-40 candidates
    per read (empty reads included), with and without a mask, and with the
    optional outputs left out: bit-exact against the oracle."""
    rng = np.random.default_rng(9)
    counts = rng.integers(0, 41, 20000)
    counts[::97] = 0
    off = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    score = rng.integers(0, 20, int(off[-1]))
    score[::11] = rng.integers(0, 2000, len(score[::11]))
    mask = (rng.random(int(off[-1])) < 0.6).astype(np.uint8)
    for m in (None, mask):
        ref = np.array(se.top_hits(score, off, m), np.int64).reshape(-1, 4)
        got = _top_hits_gpu(score, off, m)
        for k in range(4):
            np.testing.assert_array_equal(got[k], ref[:, k], err_msg=f"output {k}")
        best_only = _top_hits_gpu(score, off, m, outputs=False)
        np.testing.assert_array_equal(best_only[0], ref[:, 0])
        assert (best_only[1] == -7).all() and (best_only[3] == -7).all()


def test_top_hits_of_aligned_candidates():
    """The candidate workload (U{1..64} windows per read) aligned on each
    side: the GPU's top hits of its scores equal the oracle's of its own."""
    import torch
    from paper_1304_0681_gb300 import DeviceBatch, _swgb
    from paper_1304_0681_gb300 import stage_e
    wl = synth.generate("filter", seed=8, n_reads=250)
    b = DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets,
                                pair_read=wl.pair_read, cigar=False)
    _swgb.sw_batch_align_indexed(b.reads, b.read_offsets, b.n_reads, b.windows, b.window_offsets, b.pair_read,
                                 b.n_pairs, DEFAULT, b.score, b.end, None)
    co = torch.from_numpy(wl.cand_offsets).cuda()
    top = stage_e.top_hits(b.score, co, wl.n_reads)
    sub = wl.pair_slice(np.arange(wl.n_pairs))
    res = oracle.align_batch(sub.reads, sub.read_offsets, sub.windows, sub.window_offsets,
                             scoring=oracle.Scoring(*DEFAULT), cigar=False)
    ref = np.array(se.top_hits(res["score"], wl.cand_offsets), np.int64).reshape(-1, 4)
    for k, name in enumerate(("best_score", "best_cand", "second_score", "mapq")):
        np.testing.assert_array_equal(top[name].cpu().numpy(), ref[:, k], err_msg=name)
    # the top hit is mostly the true window, and a wrong top hit comes with
    # a lower quality (a paralog decoy scores close to the true window)
    right = ref[:, 1] == wl.true_cand
    assert right.mean() > 0.8
    assert ref[right, 3].mean() > 2 * ref[~right, 3].mean()
