"""Reference of Stage E, task iv: alignment records and splice junctions.
TEST INFRASTRUCTURE ONLY: only tests, the smoke check and the benchmark's
CPU leg may use it.

The paper (§2, Stage E) turns every SW alignment whose score passes a
threshold into an alignment record: where the read lies on the reference
(chromosome, first and last position), which part of the read aligned, and
the strand.  The same task looks for splice junctions: a long run of
consecutive deletions in the alignment marks a candidate intron, and the
candidate is kept when the intron starts and ends with the marks GT ... AG
or CT ... AC.  Junctions are counted over all batches.

Readings (the paper gives no numbers or formats for these):
- the score threshold for a record is read as score >= min_score, and
  score > 0 (an empty alignment is never a record);
- a long run of consecutive deletions is a D run of at least min_intron
  window bases;
- a window's reference coordinates are given per window: chromosome, the
  position of its first base, and its strand; the alignment covers window
  columns j_start..j_end with j_start = j_end + 1 - (M + D bases);
- a junction is (chromosome, first intron base, last intron base, strand),
  all in reference coordinates; GT...AG gives strand '+' (0), CT...AC
  strand '-' (1); other marks are not junctions;
- the alignment's quality score (one of the SW task's statistics, left
  undefined) is read per read as a mapping quality: S1 the best score of
  its candidates (the first candidate reaching it is the top hit), S2 the
  best score of the other candidates (0 without one), and quality
  min(60, floor(60 (S1 - S2) / S1)), 0 when S1 <= 0.

Every function here is a plain loop over the definition.
"""
from __future__ import annotations

import numpy as np

OP_M, OP_I, OP_D, OP_S = 0, 1, 2, 4
A, C, G, T = 0, 1, 2, 3


def runs(ops):
    """(length, op) of each BAM-encoded CIGAR run."""
    return [(int(x) >> 4, int(x) & 0xF) for x in ops]


def alignment_span(ops, i_end: int, j_end: int):
    """(i_start, j_start): first read row and first window column of the
    alignment, from its CIGAR and end cell."""
    rr = runs(ops)
    i_start = rr[0][0] if rr and rr[0][1] == OP_S else 0
    ref_len = sum(n for n, op in rr if op in (OP_M, OP_D))
    return i_start, j_end + 1 - ref_len


def record(pair, score, i_end, j_end, ops, chrom, pos, strand):
    """The alignment record of one pair, as a tuple (pair, score, chrom,
    ref_start, ref_end, read_start, read_end, strand)."""
    i_start, j_start = alignment_span(ops, i_end, j_end)
    return (int(pair), int(score), int(chrom), int(pos) + j_start, int(pos) + j_end, i_start, int(i_end),
            int(strand))


def records(score, i_end, j_end, cigars, window_chrom, window_pos, window_strand, min_score):
    """Records of every pair with score >= min_score (and > 0), in pair order."""
    out = []
    for p in range(len(score)):
        if score[p] > 0 and score[p] >= min_score:
            out.append(record(p, score[p], i_end[p], j_end[p], cigars[p], window_chrom[p], window_pos[p],
                              window_strand[p]))
    return out


def intron_strand(window, j: int, length: int):
    """0 for GT...AG, 1 for CT...AC, None otherwise (window base codes,
    intron = window[j : j + length])."""
    if length < 4:
        return None
    first = (int(window[j]), int(window[j + 1]))
    last = (int(window[j + length - 2]), int(window[j + length - 1]))
    if first == (G, T) and last == (A, G):
        return 0
    if first == (C, T) and last == (A, C):
        return 1
    return None


def pair_junctions(window, ops, j_end: int, chrom: int, pos: int, min_intron: int):
    """Junctions of one alignment: (chrom, first intron base, last intron
    base, strand) for each qualifying D run, in CIGAR order."""
    _, j = alignment_span(ops, 0, j_end)
    out = []
    for n, op in runs(ops):
        if op == OP_D:
            if n >= min_intron:
                s = intron_strand(window, j, n)
                if s is not None:
                    out.append((int(chrom), int(pos) + j, int(pos) + j + n - 1, s))
            j += n
        elif op == OP_M:
            j += n
    return out


def junction_counts(windows, window_offsets, score, j_end, cigars, window_chrom, window_pos, min_score,
                    min_intron, counts=None):
    """Add the junctions of every pair with score >= min_score (and > 0) to
    a dict {(chrom, start, end, strand): count} and return it."""
    counts = {} if counts is None else counts
    for p in range(len(score)):
        if score[p] > 0 and score[p] >= min_score:
            w = windows[window_offsets[p]:window_offsets[p + 1]]
            for key in pair_junctions(w, cigars[p], j_end[p], window_chrom[p], window_pos[p], min_intron):
                counts[key] = counts.get(key, 0) + 1
    return counts


def top_hits(score, cand_offsets, mask=None):
    """Per read: (best score, its candidate index, second-best score, mapping
    quality), over candidates with mask[p] != 0 (all without a mask); a read
    without candidates gives (-1, -1, -1, 0)."""
    out = []
    for r in range(len(cand_offsets) - 1):
        p0, p1 = int(cand_offsets[r]), int(cand_offsets[r + 1])
        cands = [(int(score[p]), p - p0) for p in range(p0, p1) if mask is None or mask[p]]
        if not cands:
            out.append((-1, -1, -1, 0))
            continue
        s1 = max(s for s, _ in cands)
        c1 = min(c for s, c in cands if s == s1)
        others = [s for s, c in cands if c != c1]
        s2 = max(others) if others else 0
        q = 0 if s1 <= 0 else min(60, (60 * (s1 - s2)) // s1)
        out.append((s1, c1, s2, q))
    return out


def cigars_of(res):
    """Per-pair CIGAR op arrays from an oracle.align_batch result."""
    off, n = res["cigar_offsets"], res["n_ops"]
    return [res["ops"][off[p]:off[p] + n[p]] for p in range(len(n))]
