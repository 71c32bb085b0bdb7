"""Pins of the Stage E task-iv oracle (alignment records, splice junctions)
against closed forms: a read split by a planted intron has a known optimal
alignment (50M L D 50M), so its record and its junction follow by hand."""
import numpy as np
import pytest

import oracle
from oracle import stage_e_oracle as se
from sw_checks import encode

SC = oracle.Scoring(5, -4, -10, -1)
POS, CHROM = 1_000_000, 7


def _read(r49, r50, seed=0):
    """100 bases over {A, C, G} with fixed bases at the split, so that the
    deletion cannot slide (a slide needs a read base equal to an intron
    mark)."""
    rng = np.random.default_rng(seed)
    r = rng.choice(list("ACG"), 100)
    r[48], r[49], r[50], r[51] = "C", r49, r50, "A"
    return "".join(r)


def _window(read, intron):
    return "T" * 20 + read[:50] + intron + read[50:] + "T" * 20


def _align(read, window):
    score, ie, je, ops = oracle.align(encode(read), encode(window), SC)
    return score, ie, je, ops


@pytest.mark.parametrize("L", [50, 120])
def test_plus_strand_junction(L):
    read = _read("A", "C")
    intron = "GT" + "T" * (L - 4) + "AG"
    w = _window(read, intron)
    score, ie, je, ops = _align(read, w)
    assert score == 500 - 10 - (L - 1)
    assert oracle.cigar_string(ops) == f"50M{L}D50M"
    assert se.alignment_span(ops, ie, je) == (0, 20)
    got = se.pair_junctions(encode(w), ops, je, CHROM, POS, min_intron=L)
    assert got == [(CHROM, POS + 70, POS + 70 + L - 1, 0)]
    assert se.pair_junctions(encode(w), ops, je, CHROM, POS, min_intron=L + 1) == []
    rec = se.record(3, score, ie, je, ops, CHROM, POS, 0)
    assert rec == (3, score, CHROM, POS + 20, POS + 20 + 100 + L - 1, 0, 99, 0)


def test_minus_strand_junction():
    read = _read("A", "G")
    L = 60
    w = _window(read, "CT" + "T" * (L - 4) + "AC")
    score, ie, je, ops = _align(read, w)
    assert oracle.cigar_string(ops) == f"50M{L}D50M"
    assert se.pair_junctions(encode(w), ops, je, CHROM, POS, 20) == [(CHROM, POS + 70, POS + 70 + L - 1, 1)]


@pytest.mark.parametrize("marks", [("AA", "TT"), ("GT", "AC"), ("CT", "AG"), ("GC", "AG")])
def test_other_marks_are_not_junctions(marks):
    # split bases unequal to the neighbouring intron marks
    r49 = next(b for b in "ACG" if b != marks[1][1])
    r50 = next(b for b in "ACG" if b != marks[0][0])
    read = _read(r49, r50)
    L = 60
    w = _window(read, marks[0] + "T" * (L - 4) + marks[1])
    score, ie, je, ops = _align(read, w)
    assert oracle.cigar_string(ops) == f"50M{L}D50M"
    assert se.pair_junctions(encode(w), ops, je, CHROM, POS, 20) == []


def test_threshold_and_counting():
    read = _read("A", "C")
    L = 50
    w = encode(_window(read, "GT" + "T" * (L - 4) + "AG"))
    r = encode(read)
    score, ie, je, ops = oracle.align(r, w, SC)
    # two copies of the pair and one unrelated pair
    junk_r, junk_w = encode("ACGT" * 5), encode("TTTT" * 30)
    js, jie, jje, jops = oracle.align(junk_r, junk_w, SC)
    windows = np.concatenate([w, w, junk_w])
    woff = np.array([0, len(w), 2 * len(w), 2 * len(w) + len(junk_w)])
    scores, ends = [score, score, js], [je, je, jje]
    cig = [ops, ops, jops]
    chrom, pos = [CHROM] * 3, [POS, POS, 5]
    c = se.junction_counts(windows, woff, scores, ends, cig, chrom, pos, min_score=score, min_intron=L)
    assert c == {(CHROM, POS + 70, POS + 70 + L - 1, 0): 2}
    # counts accumulate over calls, and the threshold is inclusive
    c = se.junction_counts(windows, woff, scores, ends, cig, chrom, pos, min_score=score, min_intron=L, counts=c)
    assert c == {(CHROM, POS + 70, POS + 70 + L - 1, 0): 4}
    assert se.junction_counts(windows, woff, scores, ends, cig, chrom, pos, score + 1, L) == {}
    recs = se.records(scores, [ie, ie, jie], ends, cig, chrom, pos, [0, 1, 0], min_score=score)
    assert [x[0] for x in recs] == [0, 1]
    assert recs[1][-1] == 1
    assert se.records(scores, [ie, ie, jie], ends, cig, chrom, pos, [0, 1, 0], min_score=score + 1) == []


def test_soft_clip_span():
    # 10 unmatched read bases before the aligned part become a leading clip
    read = "A" * 10 + _read("A", "C")
    w = _window(read[10:], "GT" + "T" * 46 + "AG")
    score, ie, je, ops = _align(read, w)
    s = oracle.cigar_string(ops)
    assert s.startswith("10S") and s.endswith("50M")
    assert se.alignment_span(ops, ie, je) == (10, 20)


def test_zero_score_is_never_a_record():
    assert se.records([0], [-1], [-1], [np.zeros(0, np.uint32)], [0], [0], [0], min_score=0) == []


def test_span_and_intron_position_with_other_gaps():
    """A 3-base window insertion before the intron (a short D run) moves the
    intron 3 columns right; a 3-base read insertion (I) moves nothing."""
    read = _read("A", "C")
    L = 50
    intron = "GT" + "T" * (L - 4) + "AG"
    # window: extra 'TTT' inside the first half (read gap -> 3D)
    w_d = "T" * 20 + read[:25] + "TTT" + read[25:50] + intron + read[50:] + "T" * 20
    score, ie, je, ops = _align(read, w_d)
    assert oracle.cigar_string(ops) == f"25M3D25M{L}D50M"
    assert se.alignment_span(ops, ie, je) == (0, 20)
    assert se.pair_junctions(encode(w_d), ops, je, CHROM, POS, L) == [(CHROM, POS + 73, POS + 73 + L - 1, 0)]
    # read: extra 'TTT' inside the first half (window gap -> 3I)
    read_i = read[:25] + "TTT" + read[25:]
    w_i = _window(read, intron)
    score, ie, je, ops = _align(read_i, w_i)
    assert oracle.cigar_string(ops) == f"25M3I25M{L}D50M"
    assert se.alignment_span(ops, ie, je) == (0, 20)
    assert se.pair_junctions(encode(w_i), ops, je, CHROM, POS, L) == [(CHROM, POS + 70, POS + 70 + L - 1, 0)]


# Top hits and mapping quality.  Hand-derived rows: (scores, mask, expected
# (best, candidate, second, quality)); quality = min(60, floor(60 (S1 - S2) / S1)).
TOP_HITS_CASES = [
    ([50], None, (50, 0, 0, 60)),                    # one candidate: no competitor
    ([50, 50], None, (50, 0, 50, 0)),                # a tie: the first wins, quality 0
    ([40, 100, 70], None, (100, 1, 70, 18)),         # 60 * 30 / 100
    ([0, 0], None, (0, 0, 0, 0)),                    # nothing aligned: quality 0
    ([], None, (-1, -1, -1, 0)),                     # no candidate
    ([100, 90, 80], [0, 1, 1], (90, 1, 80, 6)),      # masked best; 600 / 90 = 6.67
    ([100, 90], [0, 0], (-1, -1, -1, 0)),            # every candidate masked
    ([3, 1], None, (3, 0, 1, 40)),
    ([6, 7], None, (7, 1, 6, 8)),                    # 60 / 7 = 8.57
    ([9, 3, 9, 9], None, (9, 0, 9, 0)),
    ([12, 30, 29, 30], [1, 0, 1, 1], (30, 3, 29, 2)),  # 60 / 30 = 2
]


@pytest.mark.parametrize("scores,mask,expected", TOP_HITS_CASES)
def test_top_hits_hand_cases(scores, mask, expected):
    off = np.array([0, len(scores)], np.int64)
    m = None if mask is None else np.array(mask, np.uint8)
    assert se.top_hits(np.array(scores, np.int64), off, m) == [expected]


def test_top_hits_against_sorting():
    """Brute force by sorting: S1 and S2 are the two largest of the kept
    scores, the candidate is the first index of S1 (numpy's argmax), and the
    quality moves with the gap only."""
    rng = np.random.default_rng(4)
    counts = rng.integers(0, 9, 3000)
    off = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    score = rng.integers(0, 12, int(off[-1]))   # a narrow range: many ties
    mask = (rng.random(int(off[-1])) < 0.7).astype(np.uint8)
    for use_mask in (False, True):
        got = se.top_hits(score, off, mask if use_mask else None)
        for r in range(len(counts)):
            idx = np.arange(off[r], off[r + 1])
            if use_mask:
                idx = idx[mask[idx] > 0]
            if len(idx) == 0:
                assert got[r] == (-1, -1, -1, 0)
                continue
            s = score[idx]
            desc = np.sort(s)[::-1]
            s1, s2 = int(desc[0]), int(desc[1]) if len(desc) > 1 else 0
            c1 = int(idx[np.argmax(s)] - off[r])
            assert got[r][:3] == (s1, c1, s2), r
            q = got[r][3]
            assert 0 <= q <= 60
            assert (q == 0) == (s1 == 0 or s1 == s2 or 60 * (s1 - s2) < s1)
            assert (q == 60) == (s1 > 0 and 60 * (s1 - s2) >= 60 * s1)
