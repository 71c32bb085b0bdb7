"""Pins of the seeding oracle (Stages C, D, E-i, E-ii) against the paper's
worked example, a naive string search, and reads built by hand whose windows
follow from the definitions."""
import numpy as np
import pytest

import synth
from oracle import seed_oracle as so

P = so.SeedParams()


def _genome(chrom_len, seed=0):
    rng = np.random.default_rng(seed)
    codes = rng.integers(0, 4, sum(chrom_len)).astype(np.uint8)
    off = np.zeros(len(chrom_len) + 1, np.int64)
    np.cumsum(chrom_len, out=off[1:])
    return codes, off


def _windows(codes, off, read, p=P):
    w = so.seed_windows(synth.pack(codes), off, read, np.array([0, len(read)], np.int64), p)
    return [(int(s), int(a), int(b)) for s, a, b in zip(w["strand"], w["start"], w["end"])]


def test_paper_seed_example():
    """§2, Stage C: a 100-nt read gives 8 seeds from its first base and 7
    from its eighth, 15 in all, each 15 nt."""
    s = so.seed_starts(100, P)
    assert len(s) == 15
    assert s[:8] == [0, 12, 24, 36, 48, 60, 72, 84] and s[8:] == [7, 19, 31, 43, 55, 67, 79]
    assert all(x + 15 <= 100 for x in s)
    assert so.seed_starts(14, P) == [] and so.seed_starts(15, P) == [0]
    assert so.seed_starts(22, P) == [0, 7]


def test_revcomp_and_codes():
    assert so.revcomp(np.array([0, 1, 2, 3, 3], np.uint8)).tolist() == [0, 0, 1, 2, 3]
    assert so.kmer_code([0, 0, 1]) == 1 and so.kmer_code([1, 0, 0]) == 16
    assert so.kmer_code([3] * 16) == 2 ** 32 - 1


@pytest.mark.parametrize("k", [5, 8, 15, 16])
def test_exact_hits_match_naive_search(k):
    codes, off = _genome([3000, 1, 2500, 4000], seed=k)
    # a k-mer spanning the border of chromosomes 2 and 3 must not count
    border = codes[off[3] - 3:off[3] - 3 + k]
    codes[1000:1000 + k] = border  # and a genuine copy inside chromosome 0
    s = "".join("ACGT"[b] for b in codes)
    rng = np.random.default_rng(1)
    queries = [codes[q:q + k] for q in rng.integers(0, len(codes) - k, 40)] + [border]
    queries += [rng.integers(0, 4, k).astype(np.uint8) for _ in range(10)]
    hits = so.kmer_hits(synth.pack(codes), off, k, [so.kmer_code(x) for x in queries])
    for x in queries:
        t = "".join("ACGT"[b] for b in x)
        naive = [q for q in range(len(s) - k + 1) if s.startswith(t, q)
                 and np.searchsorted(off, q, side="right") == np.searchsorted(off, q + k - 1, side="right")]
        assert hits[so.kmer_code(x)].tolist() == naive
    assert (off[3] - 3) not in hits[so.kmer_code(border)].tolist()
    assert 1000 in hits[so.kmer_code(border)].tolist()


def test_exact_read_gives_one_flanked_window():
    codes, off = _genome([200_000, 100_000])
    q, m = 50_000, 100
    read = codes[q:q + m].copy()
    # the seeds cover read bases 0 .. 98 (the last seed starts at 84)
    assert _windows(codes, off, read) == [(0, q - 30, q + 98 + 30)]
    # a read from the reverse strand: strand 1 seeds its reverse complement,
    # which is the forward segment again
    assert _windows(codes, off, so.revcomp(read)) == [(1, q - 30, q + 98 + 30)]


def test_flanks_clamp_to_the_chromosome():
    codes, off = _genome([200_000, 100_000])
    c1 = int(off[1])
    read = codes[c1 + 5:c1 + 105].copy()            # 5 bases into chromosome 1, covered to c1 + 103
    assert _windows(codes, off, read) == [(0, c1, c1 + 103 + 30)]
    read = codes[c1 - 100:c1].copy()                # the last 100 bases of chromosome 0
    assert _windows(codes, off, read) == [(0, c1 - 130, c1 - 1)]


def test_spliced_read_joins_under_the_intron_limit():
    codes, off = _genome([300_000])
    a0, b0, L = 100_000, 60, 900                   # 60 bases, intron of 900, 40 bases
    read = np.concatenate([codes[a0:a0 + b0], codes[a0 + b0 + L:a0 + b0 + L + 40]])
    # seeds inside read bases 0..59 cover 0..57 (the one at 43 ends at 57);
    # seeds inside 60..99 cover 60..98 (starts 60, 67, 72, 79, 84)
    e1 = (a0 - 30, a0 + 57 + 30)
    x2 = a0 + b0 + L                               # read base 60
    e2 = (x2 - 30, x2 + 38 + 30)
    gap = e2[0] - e1[1] - 1
    assert gap == L - 58
    assert _windows(codes, off, read) == [(0, e1[0], e2[1])]
    p = so.SeedParams(max_intron=gap + 1)
    assert _windows(codes, off, read, p) == [(0, e1[0], e2[1])]
    p = so.SeedParams(max_intron=gap)              # "shorter than" the longest intron: not joined
    assert _windows(codes, off, read, p) == [(0, *e1), (0, *e2)]
    p = so.SeedParams(max_window=e2[1] - e1[0])    # the joined window would be one base too long
    assert _windows(codes, off, read, p) == [(0, *e1), (0, *e2)]


def test_repeat_filter():
    codes, off = _genome([400_000])
    seg = codes[1000:1100].copy()
    at = [50_000, 120_000, 190_000, 260_000, 330_000]
    for q in at:
        codes[q:q + 100] = seg
    read = seg.copy()
    everywhere = [(0, q - 30, q + 98 + 30) for q in [1000] + at]
    assert _windows(codes, off, read, so.SeedParams(max_hits=6)) == everywhere
    assert _windows(codes, off, read, so.SeedParams(max_hits=5)) == []


def test_merge_distance_and_cal_length_boundaries():
    off = np.array([0, 10_000, 20_000], np.int64)
    p = so.SeedParams()
    # bases strictly between: 40 - 14 - 1 = 25 < 30 -> merged; 44 - 14 - 1 = 29 -> merged; 45 -> 30 -> apart
    assert so.merge_regions([(0, 14), (40, 54)], off, p) == [(0, 54)]
    assert so.merge_regions([(44, 58), (0, 14)], off, p) == [(0, 58)]
    assert so.merge_regions([(0, 14), (45, 59)], off, p) == [(0, 14), (45, 59)]
    # never across a chromosome border
    assert so.merge_regions([(9_985, 9_999), (10_000, 10_014)], off, p) == [(9_985, 9_999), (10_000, 10_014)]
    # overlapping regions from both phases
    assert so.merge_regions([(0, 14), (7, 21), (12, 26)], off, p) == [(0, 26)]
    # a CAL spans more than min_cal_len (20) bases
    assert so.cals([(0, 19), (100, 120), (200, 214)], p) == [(100, 120)]
    assert so.extend([(100, 120)], off, p) == [(70, 150)]
    assert so.join([(0, 100), (2000, 2100), (5000, 5100)], off, p) == [(0, 2100), (5000, 5100)]
    assert so.join([(0, 100), (2101, 2200)], off, p) == [(0, 100), (2101, 2200)]
    assert so.join([(0, 100), (2100, 2200)], off, p) == [(0, 2200)]
    assert so.join([(0, 20_000)], off, p) == []  # longer than max_window on its own


def test_mutated_seeds_split_and_rejoin():
    """A 40-base stretch of mismatches kills every seed that touches it; the
    two sides become two CALs whose extended forms overlap, and the join puts
    them back into one window."""
    codes, off = _genome([200_000])
    q = 80_000
    read = codes[q:q + 150].copy()
    read[55:95] = (read[55:95] + 1) % 4
    regs = so.regions(read, so.kmer_hits(synth.pack(codes), off, 15, so.read_seed_codes(read, P)), P)
    merged = so.merge_regions(regs, off, P)
    # intact seeds: starts 0..36 and 7..31 (cover 0..50); 96..132 and 103..127 (cover 96..146);
    # 45 bases lie between the two, not fewer than 30
    assert merged == [(q + 0, q + 50), (q + 96, q + 146)]
    assert _windows(codes, off, read) == [(0, q - 30, q + 146 + 30)]


def test_generated_reads_cover_their_origin():
    """Error-free reads sampled from a generated genome: an unspliced read
    has a window on its strand that holds its whole template; a spliced read
    one that overlaps it (an exon part too short for a CAL of more than 20
    bases finds no window of its own)."""
    g = synth.genome("small", seed=2)
    rs = synth.sample_reads(g, "T2", n_reads=300, seed=4, eps=0.0, splice=0.3)
    w = so.seed_windows(g.packed, g.chrom_offsets, rs.reads, rs.read_offsets, P)
    for r in range(rs.n_reads):
        lo, hi = w["cand_offsets"][r], w["cand_offsets"][r + 1]
        a = g.chrom_offsets[rs.chrom[r]] + rs.pos[r]
        m = rs.read_offsets[r + 1] - rs.read_offsets[r]
        on = [i for i in range(lo, hi) if w["strand"][i] == rs.strand[r]]
        if rs.intron[r] >= 0:
            _, st, L, _ = g.introns[rs.intron[r]]
            last = st + L + m - (st - a) - 1
            assert any(w["start"][i] <= last and w["end"][i] >= a for i in on), r
        else:
            assert any(w["start"][i] <= a and w["end"][i] >= a + m - 1 for i in on), r
