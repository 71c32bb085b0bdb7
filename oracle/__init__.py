"""CPU oracle for the Smith-Waterman hot path -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct definition that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product path never
does.  It shares no code with the CUDA library: ``sw_oracle.c`` is a textbook
int64 Gotoh with full matrices and traceback (Stage E, task iii of the paper:
the read is aligned onto every extended / joined CAL with Smith-Waterman, which
returns the alignment, its score and its start), ``sw_brute.c`` enumerates
every alignment path of tiny inputs to pin it, and ``filter_oracle.py`` holds
the fp64 reference of the learned candidate filter.

The C sources are compiled here with gcc (``build()``); the shared object lives
next to them and is git-ignored.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from collections import namedtuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "sw_oracle.c"), os.path.join(_HERE, "sw_brute.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle_sw.so")

Scoring = namedtuple("Scoring", "match mismatch gap_open gap_extend")
#: match +5, mismatch -4, gap open -10, gap extend -1 (a gap of k costs o+(k-1)e)
DEFAULT_SCORING = Scoring(5, -4, -10, -1)

OP_M, OP_I, OP_D, OP_S = 0, 1, 2, 4
_OP_CHARS = {OP_M: "M", OP_I: "I", OP_D: "D", OP_S: "S"}

_lib = None


def build(force: bool = False, srcs=None, out: str | None = None) -> str:
    """Compile the oracle's C sources into a shared object (gcc -O2).

    ``srcs`` / ``out`` let a test compile a modified copy of the sources (a
    planted mistake) into another object."""
    srcs = list(srcs or _SRCS)
    out = out or _LIB_PATH
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, *srcs, "-lpthread"])
        os.replace(tmp, out)
    return out


def load_library(path: str):
    """ctypes handle of an oracle shared object with its signatures set."""
    lib = ctypes.CDLL(path)
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.sw_oracle_align.argtypes = [p, i64, p, i64, i64, i64, i64, i64, p, p, p, p, i64, p]
    lib.sw_oracle_align.restype = ctypes.c_int
    lib.sw_oracle_matrices.argtypes = [p, i64, p, i64, i64, i64, i64, i64, p, p, p]
    lib.sw_oracle_matrices.restype = ctypes.c_int
    lib.sw_oracle_rect_traceback.argtypes = [p, i64, p, i64, i64, i64, i64, i64, i64, i64, i64, p, i64, p, p]
    lib.sw_oracle_rect_traceback.restype = ctypes.c_int
    lib.sw_oracle_deletion_bound.argtypes = [i64, i64, i64, i64, i64]
    lib.sw_oracle_deletion_bound.restype = i64
    lib.sw_oracle_batch.argtypes = [p, p, p, p, p, i64, i64, i64, i64, i64, p, p, p, p, p, p, ctypes.c_int]
    lib.sw_oracle_batch.restype = ctypes.c_int
    lib.sw_oracle_insertion_bound.argtypes = [i64, i64, i64, i64, i64]
    lib.sw_oracle_insertion_bound.restype = i64
    lib.sw_oracle_band_traceback.argtypes = [p, i64, p, i64, i64, i64, i64, i64, i64, i64, i64, p, i64, p]
    lib.sw_oracle_band_traceback.restype = ctypes.c_int
    lib.sw_brute_tables.argtypes = [p, i64, p, i64, i64, i64, i64, i64, p, p, p]
    lib.sw_brute_tables.restype = ctypes.c_int
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _codes(x) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint8))
    return a


def cigar_capacity(m: int) -> int:
    """Runs a CIGAR of a read of length m can need: at most m M/I runs, one D
    run between or around them, and two soft clips."""
    return 2 * int(m) + 3


def align(r, w, scoring: Scoring = DEFAULT_SCORING, cigar: bool = True, lib=None):
    """Align one read against one window.  Returns (score, i_end, j_end, ops)
    with ops the BAM-encoded CIGAR (uint32 array, len << 4 | op)."""
    lib = _load(lib)
    r, w = _codes(r), _codes(w)
    out = np.zeros(3, dtype=np.int64)
    nops = np.zeros(1, dtype=np.int64)
    cap = cigar_capacity(len(r))
    ops = np.zeros(cap, dtype=np.uint32)
    rc = lib.sw_oracle_align(_ptr(r), len(r), _ptr(w), len(w), *map(int, scoring),
                             _ptr(out[0:]), _ptr(out[1:]), _ptr(out[2:]),
                             _ptr(ops) if cigar else None, cap, _ptr(nops))
    if rc != 0:
        raise RuntimeError(f"sw_oracle_align failed: {rc}")
    return int(out[0]), int(out[1]), int(out[2]), ops[: int(nops[0])].copy()


def matrices(r, w, scoring: Scoring = DEFAULT_SCORING, lib=None):
    """Filled H, E, F matrices, each (m+1) x (n+1) int64."""
    lib = _load(lib)
    r, w = _codes(r), _codes(w)
    shape = (len(r) + 1, len(w) + 1)
    H, E, F = (np.zeros(shape, dtype=np.int64) for _ in range(3))
    lib.sw_oracle_matrices(_ptr(r), len(r), _ptr(w), len(w), *map(int, scoring), _ptr(H), _ptr(E), _ptr(F))
    return H, E, F


def brute_tables(r, w, scoring: Scoring = DEFAULT_SCORING, lib=None):
    """Best path score per grid point ending with M / D / I (exhaustive)."""
    lib = _load(lib)
    r, w = _codes(r), _codes(w)
    shape = (len(r) + 1, len(w) + 1)
    bm, bd, bi = (np.zeros(shape, dtype=np.int64) for _ in range(3))
    rc = lib.sw_brute_tables(_ptr(r), len(r), _ptr(w), len(w), *map(int, scoring), _ptr(bm), _ptr(bd), _ptr(bi))
    if rc != 0:
        raise ValueError("brute force only runs for m, n <= 8")
    return bm, bd, bi


BRUTE_NEG = np.iinfo(np.int64).min // 4


def deletion_bound(i_end: int, score: int, scoring: Scoring = DEFAULT_SCORING) -> int:
    return int(_load().sw_oracle_deletion_bound(i_end, score, scoring.match, scoring.gap_open, scoring.gap_extend))


def rect_traceback(r, w, score: int, i_end: int, j_end: int, scoring: Scoring = DEFAULT_SCORING, lib=None):
    """CIGAR recomputed over the bounded rectangle only; returns (ops, j_lo)."""
    lib = _load(lib)
    r, w = _codes(r), _codes(w)
    cap = cigar_capacity(len(r))
    ops = np.zeros(cap, dtype=np.uint32)
    nops = np.zeros(1, dtype=np.int64)
    jlo = np.zeros(1, dtype=np.int64)
    rc = lib.sw_oracle_rect_traceback(_ptr(r), len(r), _ptr(w), len(w), *map(int, scoring),
                                      score, i_end, j_end, _ptr(ops), cap, _ptr(nops), _ptr(jlo))
    if rc != 0:
        raise RuntimeError(f"sw_oracle_rect_traceback failed: {rc}")
    return ops[: int(nops[0])].copy(), int(jlo[0])


def insertion_bound(i_end: int, score: int, scoring: Scoring = DEFAULT_SCORING) -> int:
    return int(_load().sw_oracle_insertion_bound(i_end, score, scoring.match, scoring.gap_open,
                                                 scoring.gap_extend))


def band_traceback(r, w, score: int, i_end: int, j_end: int, scoring: Scoring = DEFAULT_SCORING, lib=None):
    """CIGAR recomputed over the diagonal band that holds every optimal
    alignment ending at the end cell."""
    lib = _load(lib)
    r, w = _codes(r), _codes(w)
    cap = cigar_capacity(len(r))
    ops = np.zeros(cap, dtype=np.uint32)
    nops = np.zeros(1, dtype=np.int64)
    rc = lib.sw_oracle_band_traceback(_ptr(r), len(r), _ptr(w), len(w), *map(int, scoring),
                                      score, i_end, j_end, _ptr(ops), cap, _ptr(nops))
    if rc != 0:
        raise RuntimeError(f"sw_oracle_band_traceback failed: {rc}")
    return ops[: int(nops[0])].copy()


def align_batch(reads, read_offsets, windows, window_offsets, pair_read=None,
                scoring: Scoring = DEFAULT_SCORING, cigar: bool = True, threads: int | None = None, lib=None):
    """Align every pair p: read (pair_read[p] or p) against window p.

    Sequences are unpacked byte codes with CSR offsets (in bases).  Returns a
    dict with int64 arrays score, i_end, j_end and, when cigar is set, the
    CSR CIGAR (ops uint32, cigar_offsets int64, n_ops int64)."""
    lib = _load(lib)
    reads, windows = _codes(reads), _codes(windows)
    roff = np.ascontiguousarray(read_offsets, dtype=np.int64)
    woff = np.ascontiguousarray(window_offsets, dtype=np.int64)
    n_pairs = len(woff) - 1
    pr = None if pair_read is None else np.ascontiguousarray(pair_read, dtype=np.int64)
    score = np.zeros(n_pairs, np.int64)
    i_end = np.zeros(n_pairs, np.int64)
    j_end = np.zeros(n_pairs, np.int64)
    res = {"score": score, "i_end": i_end, "j_end": j_end}
    ops = cig_off = n_ops = None
    if cigar:
        rl = np.diff(roff)
        m = rl[pr] if pr is not None else rl
        cig_off = np.zeros(n_pairs + 1, np.int64)
        np.cumsum(2 * m + 3, out=cig_off[1:])
        ops = np.zeros(int(cig_off[-1]), np.uint32)
        n_ops = np.zeros(n_pairs, np.int64)
        res.update(ops=ops, cigar_offsets=cig_off, n_ops=n_ops)
    if threads is None:
        threads = os.cpu_count() or 1
    rc = lib.sw_oracle_batch(_ptr(reads), _ptr(roff), _ptr(windows), _ptr(woff),
                             _ptr(pr) if pr is not None else None, n_pairs, *map(int, scoring),
                             _ptr(score), _ptr(i_end), _ptr(j_end),
                             _ptr(ops) if cigar else None, _ptr(cig_off) if cigar else None,
                             _ptr(n_ops) if cigar else None, int(threads))
    if rc != 0:
        raise RuntimeError(f"sw_oracle_batch failed: {rc}")
    return res


def cigar_string(ops) -> str:
    """BAM-encoded ops -> text CIGAR, e.g. '50M1D50M'."""
    return "".join(f"{int(o) >> 4}{_OP_CHARS[int(o) & 0xF]}" for o in ops)


def cigar_from_string(s: str) -> np.ndarray:
    rev = {v: k for k, v in _OP_CHARS.items()}
    out, num = [], ""
    for ch in s:
        if ch.isdigit():
            num += ch
        else:
            out.append((int(num) << 4) | rev[ch])
            num = ""
    return np.array(out, dtype=np.uint32)
