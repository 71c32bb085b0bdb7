"""GPU parity of seeding (index, reads to windows, two-strand reads, window
extraction, and the whole map) against oracle/seed_oracle.py and the SW
oracle.  Windows are integers: compared exactly, field by field; k-mer
buckets as sets (the index keeps no order inside a bucket)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import seed_oracle as so

pytestmark = pytest.mark.gpu
SC = (5, -4, -10, -1)


def _torch():
    import torch
    return torch


def _params(**kw):
    from paper_1304_0681_gb300._swgb import SeedParams
    return SeedParams(**kw)


def _oparams(p):
    return so.SeedParams(k=p.k, stride=p.stride, phase=p.phase, max_hits=p.max_hits, merge_dist=p.merge_dist,
                         min_cal_len=p.min_cal_len, flank=p.flank, max_intron=p.max_intron, max_window=p.max_window)


def _index(g, k=15):
    from paper_1304_0681_gb300.seed import KmerIndex
    return KmerIndex(g.packed, g.chrom_offsets, k=k)


def _reads_dev(rs):
    torch = _torch()
    return torch.from_numpy(rs.packed_reads()).cuda(), torch.from_numpy(rs.read_offsets).cuda()


def _gpu_windows(idx, rs, p, capacity=None):
    from paper_1304_0681_gb300.seed import seed_windows
    rd, ro = _reads_dev(rs)
    w = seed_windows(idx, rd, ro, rs.n_reads, p, capacity=capacity)
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in w.items()}


def _compare(got, ref, n_reads):
    n = len(ref["start"])
    assert got["count"] == n
    np.testing.assert_array_equal(got["cand_offsets"], ref["cand_offsets"])
    np.testing.assert_array_equal(got["start"], ref["start"])
    np.testing.assert_array_equal(got["length"], ref["end"] - ref["start"] + 1)
    np.testing.assert_array_equal(got["strand"], ref["strand"])
    np.testing.assert_array_equal(got["chrom"], ref["chrom"])
    np.testing.assert_array_equal(got["pos"], ref["pos"])
    np.testing.assert_array_equal(got["pair_read"], ref["read"] + ref["strand"] * n_reads)


def _flip(code, k):
    """Oracle code (first base high) -> index code (first base low)."""
    out = 0
    for t in range(k):
        out |= ((code >> (2 * (k - 1 - t))) & 3) << (2 * t)
    return out


@pytest.mark.parametrize("k", [8, 11, 15])
def test_index_buckets_match_oracle(k):
    torch = _torch()
    # tiny and empty chromosomes: k-mers never span a border, offsets repeat
    g = synth.genome("small", seed=5, chrom_len=[20_000, 1, 0, 7, 30_000, 0, 15_000], n_introns=20,
                     rep_len=(100, 800))
    idx = _index(g, k)
    ref = so.index_buckets(g.packed, g.chrom_offsets, k)
    valid = sum(max(0, int(b - a) - k + 1) for a, b in zip(g.chrom_offsets[:-1], g.chrom_offsets[1:]))
    assert idx.n_positions == valid == sum(len(v) for v in ref.values())
    if k <= 11:
        tab = idx.table.cpu().numpy().view(np.uint32).astype(np.int64)
        pos = idx.positions[:idx.n_positions].cpu().numpy().view(np.uint32).astype(np.int64)
        lo = np.concatenate([[0], tab[:-1]])
        got = {}
        for x in np.nonzero(tab - lo)[0]:
            got[int(x)] = np.sort(pos[lo[x]:tab[x]]).tolist()
        assert got == {_flip(c, k): v.tolist() for c, v in ref.items()}
    else:
        for c, v in list(ref.items())[:400]:
            assert idx.bucket(_flip(c, k)).tolist() == v.tolist()
        rng = np.random.default_rng(0)
        for x in rng.integers(0, 4 ** k, 200):
            want = ref.get(_flip(int(x), k), np.zeros(0))  # _flip is its own inverse
            assert idx.bucket(int(x)).tolist() == want.tolist()
    del torch


@pytest.mark.parametrize("reads", ["T2", "T4"])
def test_windows_match_oracle(reads):
    g = synth.genome("small", seed=7)
    rs = synth.sample_reads(g, reads, n_reads=2500, seed=8, splice=0.15)
    idx = _index(g)
    p = _params()
    got = _gpu_windows(idx, rs, p)
    ref = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(p))
    _compare(got, ref, rs.n_reads)
    assert got["count"] > rs.n_reads  # repeats and both strands


@pytest.mark.parametrize("kw", [dict(max_hits=2), dict(merge_dist=0, min_cal_len=15), dict(max_intron=0),
                                dict(max_window=200, flank=50), dict(k=11, stride=5, phase=3, min_cal_len=11),
                                dict(k=16, stride=16, phase=8, min_cal_len=40, merge_dist=100),
                                dict(max_intron=100_000, max_window=300_000)])
def test_parameter_variants(kw):
    g = synth.genome("small", seed=9)
    rs = synth.sample_reads(g, "T2", n_reads=800, seed=10, splice=0.3,
                            lengths=((30, .1), (100, .5), (250, .3), (600, .1)))
    p = _params(**kw)
    idx = _index(g, p.k)
    got = _gpu_windows(idx, rs, p)
    ref = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(p))
    _compare(got, ref, rs.n_reads)


def test_long_hit_lists_take_the_block_path():
    """A 300-base segment copied 40 times: a 250-base read from it keeps 39
    seeds x 40 hits > 1024, more than a warp's list."""
    g = synth.genome("small", seed=11, repeat_share=0.0, n_introns=0)
    codes = g.codes().copy()
    seg = codes[1000:1300].copy()
    for t in range(40):
        q = 20_000 + t * 45_000
        codes[q:q + 300] = seg
    packed = synth.pack(codes)
    gg = synth.Genome("rep", packed, g.chrom_offsets, g.introns)
    rng = np.random.default_rng(3)
    reads = [seg[o:o + 250] for o in rng.integers(0, 50, 20)] + [codes[q:q + 250] for q in
                                                                 rng.integers(0, 1_900_000, 20)]
    roff = np.zeros(len(reads) + 1, np.int64)
    np.cumsum([len(r) for r in reads], out=roff[1:])
    rs = synth.ReadSet("rep", np.concatenate(reads), roff, *(np.zeros(len(reads), t) for t in
                                                             (np.int32, np.int64, np.int8, np.int32)))
    idx = _index(gg)
    p = _params(max_hits=64)
    got = _gpu_windows(idx, rs, p)
    ref = so.seed_windows(packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(p))
    _compare(got, ref, rs.n_reads)
    assert np.all(np.diff(got["cand_offsets"])[:20] >= 41)


def test_empty_chromosomes():
    """Chromosomes of length 0 between others: windows, chromosomes and
    chromosome positions as the oracle's."""
    g = synth.genome("small", seed=27, chrom_len=[0, 150_000, 0, 0, 120_000, 0], n_introns=30)
    rs = synth.sample_reads(g, "T2", n_reads=600, seed=28, splice=0.2)
    idx = _index(g)
    p = _params()
    _compare(_gpu_windows(idx, rs, p), so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets,
                                                        _oparams(p)), rs.n_reads)


def test_edge_cases_and_capacity_retry():
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300.seed import seed_windows
    torch = _torch()
    g = synth.genome("small", seed=12)
    idx = _index(g)
    p = _params()
    codes = g.codes()
    # empty reads, reads shorter than k, one base short of two seeds, exact reads
    reads = [np.zeros(0, np.uint8), codes[500:514], codes[600:621], codes[700:800], np.zeros(0, np.uint8),
             codes[900_000:901_024]]
    roff = np.zeros(len(reads) + 1, np.int64)
    np.cumsum([len(r) for r in reads], out=roff[1:])
    rs = synth.ReadSet("edge", np.concatenate(reads), roff, *(np.zeros(len(reads), t) for t in
                                                              (np.int32, np.int64, np.int8, np.int32)))
    ref = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(p))
    _compare(_gpu_windows(idx, rs, p), ref, rs.n_reads)
    _compare(_gpu_windows(idx, rs, p, capacity=1), ref, rs.n_reads)  # too small: retried with the count
    # no reads
    rd, ro = _reads_dev(rs)
    w = seed_windows(idx, rd, ro[:1], 0, p)
    assert w["count"] == 0 and w["cand_offsets"].cpu().tolist() == [0]
    # a read beyond the seeding limit
    long = synth.ReadSet("long", codes[:1025].copy(), np.array([0, 1025], np.int64),
                         *(np.zeros(1, t) for t in (np.int32, np.int64, np.int8, np.int32)))
    rd, ro = _reads_dev(long)
    with pytest.raises(sw.SwError) as e:
        seed_windows(idx, rd, ro, 1, p)
    assert e.value.code == -6
    torch.cuda.synchronize()


def test_two_strands_and_extract():
    torch = _torch()
    from paper_1304_0681_gb300.seed import extract_windows, two_strands
    g = synth.genome("small", seed=13)
    rs = synth.sample_reads(g, "T2", n_reads=500, seed=14, lengths=((1, .1), (17, .2), (100, .4), (333, .3)))
    rd, ro = _reads_dev(rs)
    out, off = two_strands(rd, ro, rs.n_reads)
    off = off.cpu().numpy()
    total = int(rs.read_offsets[-1])
    assert off.tolist() == rs.read_offsets[:-1].tolist() + (total + rs.read_offsets).tolist()
    got = synth.unpack(out.cpu().numpy(), 2 * total)
    want = np.concatenate([rs.reads] + [so.revcomp(rs.read(r)) for r in range(rs.n_reads)])
    np.testing.assert_array_equal(got, want)
    idx = _index(g)
    rng = np.random.default_rng(1)
    start = rng.integers(0, g.n_bases - 3000, 700).astype(np.int64)
    length = rng.integers(0, 3000, 700).astype(np.int32)
    wb, woff = extract_windows(idx, torch.from_numpy(start).cuda(), torch.from_numpy(length).cuda(), 700)
    woff = woff.cpu().numpy()
    np.testing.assert_array_equal(np.diff(woff), length)
    got = synth.unpack(wb.cpu().numpy(), int(woff[-1]))
    c = g.codes()
    np.testing.assert_array_equal(got, np.concatenate([c[a:a + n] for a, n in zip(start, length)]))


def test_map_reads_matches_oracle_alignment():
    """Seed, extract and align on the GPU; the oracle's windows aligned by
    the SW oracle give the same score and end cell for every window, and
    the same best hit per read."""
    from paper_1304_0681_gb300.seed import map_reads
    g = synth.genome("small", seed=15)
    rs = synth.sample_reads(g, "T2", n_reads=400, seed=16, splice=0.2)
    idx = _index(g)
    rd, ro = _reads_dev(rs)
    mp = map_reads(idx, rd, ro, rs.n_reads, SC)
    p = _params()
    ref = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(p))
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in mp.windows.items()}
    _compare(got, ref, rs.n_reads)
    c = g.codes()
    score = mp.score.cpu().numpy()
    end = mp.end.cpu().numpy().reshape(-1, 2)
    oscore = np.zeros(len(ref["start"]), np.int64)
    for i in range(len(ref["start"])):
        r = int(ref["read"][i])
        seq = rs.read(r) if ref["strand"][i] == 0 else so.revcomp(rs.read(r))
        s, ie, je, _ = oracle.align(seq, c[ref["start"][i]:ref["end"][i] + 1], oracle.Scoring(*SC), cigar=False)
        assert (score[i], end[i, 0], end[i, 1]) == (s, ie, je), i
        oscore[i] = s
    best = mp.best_score.cpu().numpy()
    for r in range(rs.n_reads):
        lo, hi = ref["cand_offsets"][r], ref["cand_offsets"][r + 1]
        assert best[r] == (score[lo:hi].max() if hi > lo else -1)
    # top hit, second-best score and mapping quality of every read, from the
    # oracle's own scores
    from oracle import stage_e_oracle as se
    top = np.array(se.top_hits(oscore, ref["cand_offsets"]), np.int64).reshape(-1, 4)
    for k, f in enumerate(("best_score", "best_cand", "second_score", "mapq")):
        np.testing.assert_array_equal(getattr(mp, f).cpu().numpy(), top[:, k], err_msg=f)
    # mapping accuracy: the best window of most reads holds their origin
    bc = mp.best_cand.cpu().numpy()
    hit = 0
    for r in range(rs.n_reads):
        if bc[r] < 0:
            continue
        i = ref["cand_offsets"][r] + bc[r]
        a = g.chrom_offsets[rs.chrom[r]] + rs.pos[r]
        hit += ref["strand"][i] == rs.strand[r] and ref["start"][i] <= a <= ref["end"][i]
    assert hit / rs.n_reads > 0.95


def test_full_size_sampled_parity():
    """The benchmark's workload (human-sized reference, 2M reads of 100
    bases at 1% error): a sample of reads checked one by one against the
    oracle, which scans the whole reference for their seeds."""
    g = synth.genome("human", seed=0)
    rs = synth.sample_reads(g, "T2", n_reads=2_000_000, seed=1)
    idx = _index(g)
    p = _params()
    got = _gpu_windows(idx, rs, p)
    ids = np.random.default_rng(2).choice(rs.n_reads, 24, replace=False)
    ref = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(p), read_ids=ids)
    for j, r in enumerate(ids):
        lo, hi = got["cand_offsets"][r], got["cand_offsets"][r + 1]
        rlo, rhi = ref["cand_offsets"][j], ref["cand_offsets"][j + 1]
        assert hi - lo == rhi - rlo, r
        np.testing.assert_array_equal(got["start"][lo:hi], ref["start"][rlo:rhi])
        np.testing.assert_array_equal(got["length"][lo:hi], ref["end"][rlo:rhi] - ref["start"][rlo:rhi] + 1)
        np.testing.assert_array_equal(got["strand"][lo:hi], ref["strand"][rlo:rhi])
        np.testing.assert_array_equal(got["pos"][lo:hi], ref["pos"][rlo:rhi])


def test_pipelined_batches_match_one_map():
    """Batches mapped by three workers on three streams give, read for
    read, the best hits of one map over all reads (and of the oracle)."""
    torch = _torch()
    from paper_1304_0681_gb300.seed import map_batches, map_reads
    g = synth.genome("small", seed=17)
    rs = synth.sample_reads(g, "T2", n_reads=3000, seed=18, splice=0.1,
                            lengths=((100, .6), (250, .3), (40, .1)))
    idx = _index(g)
    bounds = [0, 500, 1200, 1201, 2000, 3000]
    batches = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        sub = rs.reads[rs.read_offsets[a]:rs.read_offsets[b]]
        off = rs.read_offsets[a:b + 1] - rs.read_offsets[a]
        batches.append((torch.from_numpy(synth.pack(sub)).pin_memory(), torch.from_numpy(off).pin_memory()))
    rd, ro = _reads_dev(rs)
    whole = map_reads(idx, rd, ro, rs.n_reads, SC)
    want_score = whole.best_score.cpu().numpy()
    want_cand = whole.best_cand.cpu().numpy()
    for ns in (1, 3):
        res = map_batches(idx, batches, SC, n_streams=ns)
        np.testing.assert_array_equal(np.concatenate([r.best_score for r in res]), want_score)
        np.testing.assert_array_equal(np.concatenate([r.best_cand for r in res]), want_cand)
        np.testing.assert_array_equal(np.concatenate([r.mapq for r in res]), whole.mapq.cpu().numpy())
    ref = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(_params()),
                          read_ids=range(0, 3000, 97))
    c = g.codes()
    for j, r in enumerate(range(0, 3000, 97)):
        best = -1
        for i in range(ref["cand_offsets"][j], ref["cand_offsets"][j + 1]):
            seq = rs.read(r) if ref["strand"][i] == 0 else so.revcomp(rs.read(r))
            s, _, _, _ = oracle.align(seq, c[ref["start"][i]:ref["end"][i] + 1], oracle.Scoring(*SC), cigar=False)
            best = max(best, s)
        assert want_score[r] == best, r


def test_status_is_per_stream():
    """A capacity error on one stream is reported there and not on another."""
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300.seed import _WIN_FIELDS
    torch = _torch()
    g = synth.genome("small", seed=19)
    rs = synth.sample_reads(g, "T2", n_reads=200, seed=20)
    idx = _index(g)
    rd, ro = _reads_dev(rs)
    torch.cuda.synchronize()
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    out = {n: torch.empty(4, dtype=t, device="cuda") for n, t in _WIN_FIELDS}
    out["cand_offsets"] = torch.empty(rs.n_reads + 1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    sw._swgb.sw_seed_windows(idx.table, idx.positions, idx.chrom_offsets, idx.n_chrom, _params(), rd, ro,
                             rs.n_reads, out, 4, cnt, stream=a)
    sw._swgb.sw_sync_status(stream=b)
    with pytest.raises(sw.SwError) as e:
        sw._swgb.sw_sync_status(stream=a)
    assert e.value.code == -2
    assert int(cnt.item()) > 4


def test_stream_release_frees_and_reallocates():
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300.seed import map_reads
    torch = _torch()
    g = synth.genome("small", seed=21)
    rs = synth.sample_reads(g, "T2", n_reads=300, seed=22)
    idx = _index(g)
    rd, ro = _reads_dev(rs)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        a = map_reads(idx, rd, ro, rs.n_reads, SC).best_score.cpu().numpy()
        sw._swgb.sw_stream_release(s)
        b = map_reads(idx, rd, ro, rs.n_reads, SC).best_score.cpu().numpy()
        sw._swgb.sw_stream_release(s)
    np.testing.assert_array_equal(a, b)
    assert sw._swgb.sw_last_cuda_error()[0] == 0


def test_map_records_and_junctions_match_the_oracle_pipeline():
    """Seeded windows carry reference coordinates: the records and splice
    junctions of the whole GPU map equal the oracle pipeline's (seeding
    oracle -> SW oracle -> Stage E oracle), and the junctions are the planted
    introns the spliced reads span."""
    from oracle import stage_e_oracle as se
    from paper_1304_0681_gb300 import stage_e
    from paper_1304_0681_gb300.seed import map_reads
    g = synth.genome("small", seed=23, n_introns=300, intron=(50, 150))
    rs = synth.sample_reads(g, "T1", n_reads=1200, seed=24, splice=0.5, min_exon=35)
    idx = _index(g)
    rd, ro = _reads_dev(rs)
    tab = stage_e.JunctionTable(1 << 14)
    mp = map_reads(idx, rd, ro, rs.n_reads, SC, min_score=200, junctions=tab, min_intron=20)
    jn = tab.export()
    got_j = {(int(c), int(a), int(b), int(t)): int(k)
             for c, a, b, t, k in zip(jn["chrom"], jn["start"], jn["end"], jn["strand"], jn["count"])}
    ref = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, _oparams(_params()))
    c = g.codes()
    scores, ie, je, cig, wins = [], [], [], [], []
    for i in range(len(ref["start"])):
        r = int(ref["read"][i])
        seq = rs.read(r) if ref["strand"][i] == 0 else so.revcomp(rs.read(r))
        w = c[ref["start"][i]:ref["end"][i] + 1]
        s, a, b, ops = oracle.align(seq, w, oracle.Scoring(*SC))
        scores.append(s); ie.append(a); je.append(b); cig.append(ops); wins.append(w)
    woff = np.zeros(len(wins) + 1, np.int64)
    np.cumsum([len(w) for w in wins], out=woff[1:])
    recs = np.array(se.records(scores, ie, je, cig, ref["chrom"], ref["pos"], ref["strand"], 200),
                    np.int64).reshape(-1, 8)
    got = mp.records
    for k, col in (("pair", 0), ("score", 1), ("chrom", 2), ("ref_start", 3), ("ref_end", 4), ("read_start", 5),
                   ("read_end", 6), ("strand", 7)):
        np.testing.assert_array_equal(got[k], recs[:, col], err_msg=k)
    want_j = se.junction_counts(np.concatenate(wins), woff, scores, je, cig, ref["chrom"], ref["pos"], 200, 20)
    assert got_j == want_j
    # the junctions are planted introns: (chrom, local start, local end, strand)
    planted = {(int(ch), int(st - g.chrom_offsets[ch]), int(st - g.chrom_offsets[ch] + L - 1), int(t))
               for ch, st, L, t in g.introns}
    assert len(got_j) > 50 and set(got_j) <= planted


def test_seed_stats_count_lookups_and_hits():
    """The seeding counters: one lookup per seed of each read-strand, and
    the hits of every seed with at most max_hits of them (from the oracle's
    exact-match scan); each lookup reads at least one sector."""
    import paper_1304_0681_gb300 as sw
    g = synth.genome("small", seed=25)
    rs = synth.sample_reads(g, "T2", n_reads=700, seed=26, lengths=((40, .2), (100, .5), (250, .3)))
    idx = _index(g)
    p = _params(max_hits=8)
    _gpu_windows(idx, rs, p)
    lookups, hits, sectors = sw._swgb.sw_seed_stats()
    op = _oparams(p)
    want_lookups, want_hits, codes = 0, 0, []
    for r in range(rs.n_reads):
        for seq in (rs.read(r), so.revcomp(rs.read(r))):
            cs = so.read_seed_codes(seq, op)
            want_lookups += len(cs)
            codes.append(cs)
    table = so.kmer_hits(g.packed, g.chrom_offsets, op.k, {c for cs in codes for c in cs})
    for cs in codes:
        for c in cs:
            h = len(table.get(c, ()))
            want_hits += h if h <= op.max_hits else 0
    assert (lookups, hits) == (want_lookups, want_hits)
    assert sectors >= lookups
