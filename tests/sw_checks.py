"""Shared test helpers: independent checks of an alignment result.

These read a result (score, end cell, CIGAR) and verify it against the
strings directly, without any dynamic programming, so they can pin both the
oracle and the CUDA path."""
from __future__ import annotations

import os

import numpy as np

OP_M, OP_I, OP_D, OP_S = 0, 1, 2, 4
BASES = "ACGT"


def encode(s: str) -> np.ndarray:
    return np.array([BASES.index(c) for c in s], dtype=np.uint8)


def parse_cigar(s: str):
    ops, num = [], ""
    for ch in s:
        if ch.isdigit():
            num += ch
        else:
            ops.append((int(num), ch))
            num = ""
    return ops


def decode_ops(ops) -> list:
    return [(int(o) >> 4, "MIDNSHP=X"[int(o) & 0xF]) for o in ops]


def rescore(read, window, cigar, j_end, scoring):
    """Score of the alignment a CIGAR describes when it ends at window base
    j_end; also checks that it consumes the whole read and never leaves the
    window.  Returns (score, i_start, i_end, j_start)."""
    ma, mi, go, ge = scoring
    runs = cigar if isinstance(cigar, list) else decode_ops(cigar)
    m = len(read)
    consumed_read = sum(L for L, op in runs if op in "MIS")
    assert consumed_read == m, f"CIGAR consumes {consumed_read} read bases, read has {m}"
    win_span = sum(L for L, op in runs if op in "MD")
    j = j_end - win_span + 1
    assert j >= 0, "alignment starts before the window"
    i = 0
    score = 0
    i_start = None
    j_start = j
    for L, op in runs:
        if op == "S":
            i += L
        elif op == "M":
            if i_start is None:
                i_start = i
            for _ in range(L):
                score += ma if read[i] == window[j] else mi
                i += 1
                j += 1
        elif op == "I":
            score += go + (L - 1) * ge
            i += L
        elif op == "D":
            score += go + (L - 1) * ge
            j += L
    assert j - 1 == j_end
    i_end = i - 1 - sum(L for L, op in runs[-1:] if op == "S")
    return score, i_start, i_end, j_start


def load_golden(name: str):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            r, w, ma, mi, go, ge, sc, ie, je, cg = line.split()
            rows.append(dict(read=r, window=w, scoring=(int(ma), int(mi), int(go), int(ge)), score=int(sc),
                             i_end=int(ie), j_end=int(je), cigar="" if cg == "*" else cg))
    return rows
