"""Reference of seeding: reads to candidate windows.  TEST INFRASTRUCTURE
ONLY: only tests, the smoke check and the benchmark's CPU leg may use it.

The paper's Stages C and D and the first two tasks of Stage E turn a read
into the reference windows Smith-Waterman aligns it against:

  Stage C   the read is split into overlapping seeds of 15 bases, taken at
            two phases (a 100-base read gives 8 seeds from its first base and
            7 more from its eighth); each seed is mapped exactly (no errors)
            onto the reference, and every hit is a region;
  Stage D   the regions of a read that lie less than a distance apart are
            merged, and a merged region longer than a threshold is a
            candidate alignment location (CAL);
  Stage E   (i) each CAL is extended by 30 bases on both sides; (ii)
            extended CALs closer to each other than the longest known intron
            are joined into one window, chains of more than two included.

Readings (the paper leaves these open; the CUDA path takes the same ones):
- seeds start at 0, stride, 2 stride, ... and at phase, phase + stride, ...
  wherever k bases fit in the read; k = 15, phase = 7 (the eighth base) and
  stride = 12 give the paper's 8 + 7 seeds for 100 bases;
- a seed hits reference position q when bases q .. q+k-1 lie in one
  chromosome and equal the seed; a seed with more than max_hits hits is
  dropped (repeats);
- the reverse strand is the same procedure applied to the read's reverse
  complement; its windows pair that reverse complement with the forward
  reference (strand 1);
- a region is the reference interval [q, q + k - 1]; regions of one read and
  strand are merged in reference order when the bases strictly between a
  region and the merged region before it number fewer than merge_dist and
  both lie in one chromosome;
- a merged region is a CAL when it spans more than min_cal_len bases;
- extension is clamped to the chromosome;
- in reference order, an extended CAL joins the window before it when they
  lie in one chromosome, fewer than max_intron bases lie strictly between
  them, and the joined window spans at most max_window bases; otherwise it
  starts a new window; an extended CAL longer than max_window on its own is
  dropped;
- windows come out per read, strand 0 before strand 1, in reference order.

Coordinates are global positions in the back-to-back chromosomes; a window
also carries its chromosome and its chromosome-local start.  Every step
below is a plain loop over its definition.  The exact-match scan is plain C
(``seed_hits.c``); everything else is here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seed_hits.c")
_LIB_PATH = os.path.join(_HERE, "libseed_hits.so")
_lib = None


@dataclass(frozen=True)
class SeedParams:
    k: int = 15
    stride: int = 12
    phase: int = 7
    max_hits: int = 64
    merge_dist: int = 30
    min_cal_len: int = 20
    flank: int = 30
    max_intron: int = 2000
    max_window: int = 16384


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.seed_hits.argtypes = [p, p, i32, i32, p, i64, p, p, p]
        lib.seed_hits.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def seed_starts(m: int, p: SeedParams = SeedParams()):
    """Start of every seed of an m-base read: first phase, then second."""
    out = []
    for first in (0, p.phase):
        s = first
        while s + p.k <= m:
            out.append(s)
            s += p.stride
    return out


def revcomp(codes) -> np.ndarray:
    """Reverse complement of base codes (A=0 C=1 G=2 T=3)."""
    return (3 - np.asarray(codes, np.uint8)[::-1]).astype(np.uint8)


def kmer_code(codes) -> int:
    """Code of a k-mer with its first base in the most significant bits."""
    x = 0
    for b in codes:
        x = (x << 2) | int(b)
    return x


def kmer_hits(packed, chrom_offsets, k: int, codes) -> dict:
    """{code: ascending numpy array of the positions where it occurs}."""
    lib = _load()
    uniq = np.unique(np.asarray(list(codes), np.uint32))
    off = np.ascontiguousarray(chrom_offsets, np.int64)
    packed = np.ascontiguousarray(packed, np.uint8)
    cnt = np.zeros(max(len(uniq), 1), np.int64)
    rc = lib.seed_hits(_ptr(packed), _ptr(off), len(off) - 1, k, _ptr(uniq), len(uniq), _ptr(cnt), None, None)
    if rc:
        raise RuntimeError(f"seed_hits failed: {rc}")
    cnt = cnt[:len(uniq)]
    base = np.zeros(len(uniq) + 1, np.int64)
    np.cumsum(cnt, out=base[1:])
    pos = np.zeros(max(int(base[-1]), 1), np.int64)
    rc = lib.seed_hits(_ptr(packed), _ptr(off), len(off) - 1, k, _ptr(uniq), len(uniq), None, _ptr(base),
                       _ptr(pos))
    if rc:
        raise RuntimeError(f"seed_hits failed: {rc}")
    return {int(c): pos[base[i]:base[i + 1]].copy() for i, c in enumerate(uniq)}


def chrom_of(chrom_offsets, q: int) -> int:
    """Chromosome holding global position q."""
    c = 0
    while chrom_offsets[c + 1] <= q:
        c += 1
    return c


def regions(seq, hits: dict, p: SeedParams):
    """Stage C: the reference intervals [q, q + k - 1] of the seeds' hits."""
    out = []
    for s in seed_starts(len(seq), p):
        h = hits.get(kmer_code(seq[s:s + p.k]), ())
        if len(h) > p.max_hits:
            continue
        out.extend((int(q), int(q) + p.k - 1) for q in h)
    return out


def merge_regions(regs, chrom_offsets, p: SeedParams):
    """Stage D, first step: merge regions in reference order."""
    merged = []
    for a, b in sorted(regs):
        if merged:
            ma, mb = merged[-1]
            if a - mb - 1 < p.merge_dist and chrom_of(chrom_offsets, a) == chrom_of(chrom_offsets, ma):
                merged[-1] = (ma, max(mb, b))
                continue
        merged.append((a, b))
    return merged


def cals(merged, p: SeedParams):
    """Stage D, second step: merged regions longer than min_cal_len."""
    return [(a, b) for a, b in merged if b - a + 1 > p.min_cal_len]


def extend(cal_list, chrom_offsets, p: SeedParams):
    """Stage E, task i: flank bases on both sides, within the chromosome."""
    out = []
    for a, b in cal_list:
        c = chrom_of(chrom_offsets, a)
        out.append((max(a - p.flank, int(chrom_offsets[c])), min(b + p.flank, int(chrom_offsets[c + 1]) - 1)))
    return out


def join(ext, chrom_offsets, p: SeedParams):
    """Stage E, task ii: join extended CALs closer than the longest intron."""
    out = []
    for a, b in ext:
        if b - a + 1 > p.max_window:
            continue
        if out:
            ja, jb = out[-1]
            if (chrom_of(chrom_offsets, a) == chrom_of(chrom_offsets, ja) and a - jb - 1 < p.max_intron
                    and max(jb, b) - ja + 1 <= p.max_window):
                out[-1] = (ja, max(jb, b))
                continue
        out.append((a, b))
    return out


def strand_windows(seq, hits: dict, chrom_offsets, p: SeedParams):
    """Windows (global start, global end) of one read sequence."""
    m = merge_regions(regions(seq, hits, p), chrom_offsets, p)
    return join(extend(cals(m, p), chrom_offsets, p), chrom_offsets, p)


def read_seed_codes(seq, p: SeedParams):
    return [kmer_code(seq[s:s + p.k]) for s in seed_starts(len(seq), p)]


def seed_windows(packed, chrom_offsets, reads, read_offsets, p: SeedParams = SeedParams(), read_ids=None,
                 hits: dict | None = None):
    """Windows of the given reads (all by default), as a dict of numpy
    arrays in output order: read, strand, start, end (global, inclusive),
    chrom, pos (chromosome-local start), and the per-read candidate offsets
    (over the given reads)."""
    ids = range(len(read_offsets) - 1) if read_ids is None else read_ids
    seqs = []
    for r in ids:
        f = np.asarray(reads[read_offsets[r]:read_offsets[r + 1]], np.uint8)
        seqs.append((r, f, revcomp(f)))
    if hits is None:
        codes = set()
        for _, f, rc in seqs:
            codes.update(read_seed_codes(f, p))
            codes.update(read_seed_codes(rc, p))
        hits = kmer_hits(packed, chrom_offsets, p.k, codes)
    rows, cand = [], [0]
    for r, f, rc in seqs:
        for strand, seq in ((0, f), (1, rc)):
            for a, b in strand_windows(seq, hits, chrom_offsets, p):
                c = chrom_of(chrom_offsets, a)
                rows.append((r, strand, a, b, c, a - int(chrom_offsets[c])))
        cand.append(len(rows))
    a = np.array(rows, np.int64).reshape(-1, 6)
    return {"read": a[:, 0], "strand": a[:, 1], "start": a[:, 2], "end": a[:, 3], "chrom": a[:, 4],
            "pos": a[:, 5], "cand_offsets": np.array(cand, np.int64)}


def index_buckets(packed, chrom_offsets, k: int):
    """{code: ascending positions} of every k-mer of the reference (small
    references only: the table of all k-mers)."""
    G = int(chrom_offsets[-1])
    codes = set()
    # every code that occurs is a candidate: read them off the reference
    base = ((np.asarray(packed, np.uint8)[np.arange(G) >> 2] >> (2 * (np.arange(G) & 3))) & 3).astype(np.int64)
    for c in range(len(chrom_offsets) - 1):
        lo, hi = int(chrom_offsets[c]), int(chrom_offsets[c + 1])
        for q in range(lo, hi - k + 1):
            codes.add(kmer_code(base[q:q + k]))
    return kmer_hits(packed, chrom_offsets, k, codes)
