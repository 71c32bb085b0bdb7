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
