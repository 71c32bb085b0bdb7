"""Seeded synthetic (read, candidate window) workloads.

This module only makes inputs -- it holds none of the alignment arithmetic --
and is the one piece both the oracle and the CUDA path consume.  The C
generator (``synth.c``) is compiled with gcc on first use.

Workload recipes (the paper's datasets -- dwgsim-simulated 100/250 nt reads at
0.1% / 1% error with 30% indels, mapped against a genome -- are not available,
so these stand in for the candidate windows its Stage E receives):

``parity``      1,000 pairs; reads 100 bp; windows 150 bp holding the read
                mutated (2% substitutions, 0.5% indels of length 1-3) at a
                uniform offset in random flanks.
``throughput``  1,000,000 pairs; reads 100 bp; windows 200 bp; same mutation
                model; 20% of windows are random decoys.
``uneven``      2,000,000 pairs; read length from {75:.20, 100:.30, 150:.25,
                250:.15, 400:.07, 800:.03}; window = flank U(20,100) + mutated
                read + flank U(20,100); divergence U(0.5%, 5%), 80% of events
                substitutions and 20% indels; 10% of reads spliced: the window
                holds the two halves of the mutated read around a random intron
                of U{50..2000} bp that starts with GT and ends with AG.
``filter``      500,000 reads of 150 bp, each with U{1..64} candidate windows
                of 250 bp: one true window at U(1%, 3%) divergence, the other
                candidates split 50/50 between paralog-like decoys (the read
                mutated at U(5%, 20%)) and random windows.
``fullmix``     reads as ``uneven`` with 15% spliced and U{1..32} candidates:
                one true at U(1%, 5%), decoys paralog U(5%, 20%) or random.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_CORE = os.path.join(_HERE, "synth_core.h")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")

KIND_TRUE, KIND_PARALOG, KIND_RANDOM = 0, 1, 2


class SynthSpec(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_reads", ctypes.c_int64),
        ("n_len", ctypes.c_int32),
        ("len_val", ctypes.c_int32 * 8),
        ("len_w", ctypes.c_double * 8),
        ("cand_min", ctypes.c_int32),
        ("cand_max", ctypes.c_int32),
        ("win_len", ctypes.c_int32),
        ("flank_min", ctypes.c_int32),
        ("flank_max", ctypes.c_int32),
        ("div_lo", ctypes.c_double),
        ("div_hi", ctypes.c_double),
        ("indel_share", ctypes.c_double),
        ("decoy_random", ctypes.c_double),
        ("paralog_share", ctypes.c_double),
        ("par_lo", ctypes.c_double),
        ("par_hi", ctypes.c_double),
        ("splice_frac", ctypes.c_double),
        ("intron_min", ctypes.c_int32),
        ("intron_max", ctypes.c_int32),
        ("first_read", ctypes.c_int64),
    ]


def _spec(seed, n_reads, lengths, cand=(1, 1), win_len=0, flanks=(20, 100), div=(0.025, 0.025),
          indel_share=0.2, decoy_random=0.0, paralog_share=0.5, par=(0.05, 0.20), splice=0.0,
          intron=(50, 2000)) -> SynthSpec:
    s = SynthSpec()
    s.seed = seed
    s.n_reads = n_reads
    s.n_len = len(lengths)
    for k, (v, w) in enumerate(lengths):
        s.len_val[k] = v
        s.len_w[k] = w
    s.cand_min, s.cand_max = cand
    s.win_len = win_len
    s.flank_min, s.flank_max = flanks
    s.div_lo, s.div_hi = div
    s.indel_share = indel_share
    s.decoy_random = decoy_random
    s.paralog_share = paralog_share
    s.par_lo, s.par_hi = par
    s.splice_frac = splice
    s.intron_min, s.intron_max = intron
    return s


UNEVEN_LENGTHS = ((75, .20), (100, .30), (150, .25), (250, .15), (400, .07), (800, .03))


def spec_for(name: str, seed: int = 0, n_reads: int | None = None) -> SynthSpec:
    """The generator parameters of a named workload (n_reads overrides the size)."""
    if name == "parity":
        return _spec(seed, n_reads or 1000, ((100, 1.0),), win_len=150, div=(0.025, 0.025))
    if name == "throughput":
        return _spec(seed, n_reads or 1_000_000, ((100, 1.0),), win_len=200, div=(0.025, 0.025),
                     decoy_random=0.2)
    if name == "uneven":
        return _spec(seed, n_reads or 2_000_000, UNEVEN_LENGTHS, flanks=(20, 100), div=(0.005, 0.05),
                     splice=0.10, intron=(50, 2000))
    if name == "filter":
        return _spec(seed, n_reads or 500_000, ((150, 1.0),), cand=(1, 64), win_len=250, div=(0.01, 0.03),
                     paralog_share=0.5, par=(0.05, 0.20))
    if name == "fullmix":
        return _spec(seed, n_reads or 10_000_000, UNEVEN_LENGTHS, cand=(1, 32), flanks=(20, 100),
                     div=(0.01, 0.05), paralog_share=0.5, par=(0.05, 0.20), splice=0.15, intron=(50, 2000))
    raise KeyError(name)


_lib = None


def _stale(lib: str, *srcs: str) -> bool:
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    """Compile the host generator (gcc; no contraction of floating-point
    expressions, so its uniforms compare as the device generator's do)."""
    if force or _stale(_LIB_PATH, _SRC, _CORE):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC,
                               "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.synth_headers.argtypes = [ctypes.POINTER(SynthSpec), p, p, ctypes.c_int]
        lib.synth_window_lengths.argtypes = [ctypes.POINTER(SynthSpec), p, p, ctypes.c_int]
        lib.synth_fill.argtypes = [ctypes.POINTER(SynthSpec), p, p, p, p, p, p, p, ctypes.c_int]
        lib.synth_pack.argtypes = [p, i64, p]
        lib.synth_pack.restype = None
        lib.synth_unpack.argtypes = [p, i64, p]
        lib.synth_unpack.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def packed_nbytes(n_bases: int) -> int:
    """Bytes of a 2-bit packed buffer of n_bases, rounded up to 16 bytes so
    that aligned 16-byte loads of the last bases stay inside the buffer."""
    return ((int(n_bases) + 3) // 4 + 15) // 16 * 16


def pack(codes: np.ndarray) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.zeros(packed_nbytes(len(codes)), dtype=np.uint8)
    _load().synth_pack(_ptr(codes), len(codes), _ptr(out))
    return out


def unpack(packed: np.ndarray, n_bases: int) -> np.ndarray:
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    out = np.zeros(n_bases, dtype=np.uint8)
    _load().synth_unpack(_ptr(packed), int(n_bases), _ptr(out))
    return out


@dataclass
class Workload:
    """Reads and candidate windows in CSR form (offsets in bases).

    Pair p aligns read ``pair_read[p]`` against window p.  Read r owns the
    candidate pairs ``cand_offsets[r] .. cand_offsets[r+1]``."""
    name: str
    reads: np.ndarray            # uint8 codes, all reads back to back
    read_offsets: np.ndarray     # int64, n_reads + 1
    windows: np.ndarray          # uint8 codes, all windows back to back
    window_offsets: np.ndarray   # int64, n_pairs + 1
    pair_read: np.ndarray        # int64, n_pairs
    cand_offsets: np.ndarray     # int64, n_reads + 1
    kinds: np.ndarray            # uint8, n_pairs: 0 true, 1 paralog, 2 random
    true_cand: np.ndarray        # int32, n_reads: index of the true candidate
    _packed: dict = field(default_factory=dict, repr=False)

    @property
    def n_reads(self) -> int:
        return len(self.read_offsets) - 1

    @property
    def n_pairs(self) -> int:
        return len(self.window_offsets) - 1

    @property
    def read_lengths(self) -> np.ndarray:
        return np.diff(self.read_offsets)

    @property
    def window_lengths(self) -> np.ndarray:
        return np.diff(self.window_offsets)

    @property
    def pair_read_lengths(self) -> np.ndarray:
        return self.read_lengths[self.pair_read]

    def cells(self) -> int:
        """Sum of m * n over pairs: the DP cells one full pass updates."""
        return int(np.sum(self.pair_read_lengths.astype(np.int64) * self.window_lengths))

    def packed_reads(self) -> np.ndarray:
        if "reads" not in self._packed:
            self._packed["reads"] = pack(self.reads)
        return self._packed["reads"]

    def packed_windows(self) -> np.ndarray:
        if "windows" not in self._packed:
            self._packed["windows"] = pack(self.windows)
        return self._packed["windows"]

    def pair_slice(self, pairs: np.ndarray) -> "Workload":
        """A workload holding only the given pairs (one read copy per pair)."""
        pairs = np.asarray(pairs, dtype=np.int64)
        rl = self.pair_read_lengths[pairs]
        wl = self.window_lengths[pairs]
        roff = np.zeros(len(pairs) + 1, np.int64)
        np.cumsum(rl, out=roff[1:])
        woff = np.zeros(len(pairs) + 1, np.int64)
        np.cumsum(wl, out=woff[1:])
        reads = np.concatenate([self.reads[self.read_offsets[r]:self.read_offsets[r + 1]]
                                for r in self.pair_read[pairs]]) if len(pairs) else np.zeros(0, np.uint8)
        wins = np.concatenate([self.windows[self.window_offsets[p]:self.window_offsets[p + 1]]
                               for p in pairs]) if len(pairs) else np.zeros(0, np.uint8)
        return Workload(self.name + "[slice]", reads, roff, wins, woff, np.arange(len(pairs), dtype=np.int64),
                        np.arange(len(pairs) + 1, dtype=np.int64), self.kinds[pairs].copy(),
                        np.zeros(len(pairs), np.int32))


    def read_slice(self, lo: int, hi: int) -> "Workload":
        """Reads lo .. hi with all of their candidate pairs (offsets rebased)."""
        p0, p1 = int(self.cand_offsets[lo]), int(self.cand_offsets[hi])
        r0, r1 = int(self.read_offsets[lo]), int(self.read_offsets[hi])
        w0, w1 = int(self.window_offsets[p0]), int(self.window_offsets[p1])
        return Workload(f"{self.name}[{lo}:{hi}]", self.reads[r0:r1].copy(), self.read_offsets[lo:hi + 1] - r0,
                        self.windows[w0:w1].copy(), self.window_offsets[p0:p1 + 1] - w0,
                        self.pair_read[p0:p1] - lo, self.cand_offsets[lo:hi + 1] - p0,
                        self.kinds[p0:p1].copy(), self.true_cand[lo:hi].copy())


def generate(name: str, seed: int = 0, n_reads: int | None = None, threads: int | None = None,
             first_read: int = 0) -> Workload:
    """Generate a named workload deterministically (independent of threads).

    Every read and its candidates depend only on (seed, read index), so
    ``first_read=R, n_reads=n`` gives reads R .. R+n-1 of any larger set of
    the same seed (offsets rebased to 0)."""
    lib = _load()
    spec = spec_for(name, seed, n_reads)
    spec.first_read = first_read
    nt = threads or min(os.cpu_count() or 1, 32)
    nr = int(spec.n_reads)
    read_len = np.zeros(nr, np.int32)
    n_cand = np.zeros(nr, np.int32)
    rc = lib.synth_headers(ctypes.byref(spec), _ptr(read_len), _ptr(n_cand), nt)
    if rc:
        raise RuntimeError(f"synth_headers failed: {rc}")
    cand_off = np.zeros(nr + 1, np.int64)
    np.cumsum(n_cand, out=cand_off[1:])
    n_pairs = int(cand_off[-1])
    win_len = np.zeros(n_pairs, np.int32)
    rc = lib.synth_window_lengths(ctypes.byref(spec), _ptr(cand_off), _ptr(win_len), nt)
    if rc:
        raise RuntimeError(f"synth_window_lengths failed: {rc}")
    read_off = np.zeros(nr + 1, np.int64)
    np.cumsum(read_len, out=read_off[1:])
    win_off = np.zeros(n_pairs + 1, np.int64)
    np.cumsum(win_len, out=win_off[1:])
    reads = np.zeros(int(read_off[-1]), np.uint8)
    wins = np.zeros(int(win_off[-1]), np.uint8)
    kinds = np.zeros(n_pairs, np.uint8)
    true_cand = np.zeros(nr, np.int32)
    rc = lib.synth_fill(ctypes.byref(spec), _ptr(cand_off), _ptr(read_off), _ptr(win_off),
                        _ptr(reads), _ptr(wins), _ptr(kinds), _ptr(true_cand), nt)
    if rc:
        raise RuntimeError(f"synth_fill failed: {rc}")
    pair_read = np.repeat(np.arange(nr, dtype=np.int64), n_cand)
    return Workload(name, reads, read_off, wins, win_off, pair_read, cand_off, kinds, true_cand)


# --------------------------------------------------------------------------
# The same generator on the device (synth_gpu.cu includes synth_core.h as
# synth.c does), for workloads too large to generate on the host.

_GPU_SRC = os.path.join(_HERE, "synth_gpu.cu")
_GPU_LIB_PATH = os.path.join(_HERE, "libsynth_gpu.so")
_gpu_lib = None


def build_gpu(force: bool = False) -> str:
    """Compile the device generator (nvcc, sm_103a, -fmad=false so that its
    double expressions round as the host generator's do)."""
    if force or _stale(_GPU_LIB_PATH, _GPU_SRC, _CORE):
        tmp = _GPU_LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([os.environ.get("NVCC", "nvcc"), "-gencode", "arch=compute_103a,code=sm_103a",
                               "-O3", "-fmad=false", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
                               "-o", tmp, _GPU_SRC])
        os.replace(tmp, _GPU_LIB_PATH)
    return _GPU_LIB_PATH


def _load_gpu():
    global _gpu_lib
    if _gpu_lib is None:
        lib = ctypes.CDLL(build_gpu())
        p, sp = ctypes.c_void_p, ctypes.POINTER(SynthSpec)
        lib.synth_gpu_headers.argtypes = [sp, p, p, p]
        lib.synth_gpu_reads.argtypes = [sp, p, p, p, p]
        lib.synth_gpu_windows.argtypes = [sp, p, p, ctypes.c_int64, p, p, p, p, p]
        _gpu_lib = lib
    return _gpu_lib


@dataclass
class DeviceWorkload:
    """A workload generated on the device: the arrays of Workload as CUDA
    tensors, reads and windows 2-bit packed (synth_pack's layout)."""
    name: str
    reads: "torch.Tensor"           # uint8, packed, packed_nbytes(total read bases)
    read_offsets: "torch.Tensor"    # int64, n_reads + 1
    windows: "torch.Tensor"         # uint8, packed
    window_offsets: "torch.Tensor"  # int64, n_pairs + 1
    pair_read: "torch.Tensor"       # int64, n_pairs
    cand_offsets: "torch.Tensor"    # int64, n_reads + 1
    kinds: "torch.Tensor"           # uint8, n_pairs
    true_cand: "torch.Tensor"       # int32, n_reads

    @property
    def n_reads(self) -> int:
        return self.read_offsets.numel() - 1

    @property
    def n_pairs(self) -> int:
        return self.window_offsets.numel() - 1

    @property
    def pair_read_lengths(self):
        return (self.read_offsets[1:] - self.read_offsets[:-1])[self.pair_read]

    def cells(self) -> int:
        """Sum of m * n over pairs."""
        return int(((self.window_offsets[1:] - self.window_offsets[:-1]) * self.pair_read_lengths).sum().item())


def generate_device(name: str, seed: int = 0, n_reads: int | None = None, device="cuda",
                    first_read: int = 0) -> DeviceWorkload:
    """generate() on the device: the same workload, packed, without a host
    copy."""
    import torch

    lib = _load_gpu()
    spec = spec_for(name, seed, n_reads)
    spec.first_read = first_read
    nr = int(spec.n_reads)
    dev = torch.device(device)
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def call(rc, what):
        if rc:
            raise RuntimeError(f"{what} failed: {rc}")

    def cumsum0(x):
        out = torch.zeros(x.numel() + 1, dtype=torch.int64, device=dev)
        torch.cumsum(x.to(torch.int64), 0, out=out[1:])
        return out

    read_len = torch.empty(nr, dtype=torch.int32, device=dev)
    n_cand = torch.empty(nr, dtype=torch.int32, device=dev)
    call(lib.synth_gpu_headers(ctypes.byref(spec), read_len.data_ptr(), n_cand.data_ptr(), st), "synth_gpu_headers")
    cand_off = cumsum0(n_cand)
    read_off = cumsum0(read_len)
    n_pairs = int(cand_off[-1].item())
    pair_read = torch.repeat_interleave(torch.arange(nr, dtype=torch.int64, device=dev), n_cand.to(torch.int64),
                                        output_size=n_pairs)
    win_len = torch.empty(n_pairs, dtype=torch.int32, device=dev)
    call(lib.synth_gpu_windows(ctypes.byref(spec), pair_read.data_ptr(), cand_off.data_ptr(), n_pairs, None,
                               win_len.data_ptr(), None, None, st), "synth_gpu_windows (lengths)")
    win_off = cumsum0(win_len)
    del win_len
    reads = torch.zeros(packed_nbytes(int(read_off[-1].item())), dtype=torch.uint8, device=dev)
    wins = torch.zeros(packed_nbytes(int(win_off[-1].item())), dtype=torch.uint8, device=dev)
    kinds = torch.empty(n_pairs, dtype=torch.uint8, device=dev)
    true_cand = torch.empty(nr, dtype=torch.int32, device=dev)
    call(lib.synth_gpu_reads(ctypes.byref(spec), read_off.data_ptr(), reads.data_ptr(), true_cand.data_ptr(), st),
         "synth_gpu_reads")
    call(lib.synth_gpu_windows(ctypes.byref(spec), pair_read.data_ptr(), cand_off.data_ptr(), n_pairs,
                               win_off.data_ptr(), None, wins.data_ptr(), kinds.data_ptr(), st),
         "synth_gpu_windows (fill)")
    return DeviceWorkload(name, reads, read_off, wins, win_off, pair_read, cand_off, kinds, true_cand)


def random_pairs(n_pairs: int, m_range, n_range, seed: int = 0, alphabet: int = 4) -> Workload:
    """Independent uniform pairs with lengths drawn from the given inclusive
    ranges (edge-case and tie-heavy test inputs; alphabet < 4 forces ties)."""
    rng = np.random.Generator(np.random.Philox(seed))
    ml = rng.integers(m_range[0], m_range[1] + 1, n_pairs)
    nl = rng.integers(n_range[0], n_range[1] + 1, n_pairs)
    roff = np.zeros(n_pairs + 1, np.int64)
    np.cumsum(ml, out=roff[1:])
    woff = np.zeros(n_pairs + 1, np.int64)
    np.cumsum(nl, out=woff[1:])
    reads = rng.integers(0, alphabet, int(roff[-1])).astype(np.uint8)
    wins = rng.integers(0, alphabet, int(woff[-1])).astype(np.uint8)
    return Workload("random", reads, roff, wins, woff, np.arange(n_pairs, dtype=np.int64),
                    np.arange(n_pairs + 1, dtype=np.int64), np.full(n_pairs, KIND_RANDOM, np.uint8),
                    np.zeros(n_pairs, np.int32))


# --------------------------------------------------------------------------
# Reference genomes and reads sampled from them (the inputs of seeding).

class GenomeSpec(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_chrom", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("repeat_share", ctypes.c_double),
        ("rep_len_min", ctypes.c_int32),
        ("rep_len_max", ctypes.c_int32),
        ("rep_copies_min", ctypes.c_int32),
        ("rep_copies_max", ctypes.c_int32),
        ("rep_div_lo", ctypes.c_double),
        ("rep_div_hi", ctypes.c_double),
        ("n_introns", ctypes.c_int64),
        ("intron_min", ctypes.c_int32),
        ("intron_max", ctypes.c_int32),
        ("margin", ctypes.c_int32),
        ("pad1", ctypes.c_int32),
    ]


class ReadsSpec(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_reads", ctypes.c_int64),
        ("n_len", ctypes.c_int32),
        ("len_val", ctypes.c_int32 * 8),
        ("pad0", ctypes.c_int32),
        ("len_w", ctypes.c_double * 8),
        ("eps", ctypes.c_double),
        ("indel_share", ctypes.c_double),
        ("splice_frac", ctypes.c_double),
        ("min_exon", ctypes.c_int32),
        ("pad1", ctypes.c_int32),
    ]


#: Chromosome lengths (Mb) of a human-sized genome: 22 autosomes, X and Y.
HUMAN_MB = (249, 243, 198, 191, 181, 171, 159, 146, 141, 136, 135, 134, 115, 107, 102, 90, 81, 78, 59, 63, 48, 51,
            155, 59)

GENOMES = {
    # 3.1 Gb in 24 chromosomes; 5% in repeat families of 300-6,000 bp with
    # 2-20 copies at 0-8% divergence; 200,000 introns of 50-2,000 bp.
    "human": dict(chrom_len=[x * 1_000_000 for x in HUMAN_MB], repeat_share=0.05, rep_len=(300, 6000),
                  rep_copies=(2, 20), rep_div=(0.0, 0.08), n_introns=200_000, intron=(50, 2000)),
    # a quarter of "human" (774 Mb, same 24 chromosomes scaled, 50k introns):
    # with k = 14 seeds it gives the random hits per seed of "human" with
    # k = 15, in a quarter of the device memory (profiling captures)
    "quarter": dict(chrom_len=[x * 250_000 for x in HUMAN_MB], repeat_share=0.05, rep_len=(300, 6000),
                    rep_copies=(2, 20), rep_div=(0.0, 0.08), n_introns=50_000, intron=(50, 2000)),
    # 64 Mb in 8 chromosomes, same feature mix (full-size sampled parity
    # checks that the oracle can still scan).
    "medium": dict(chrom_len=[8_000_000] * 8, repeat_share=0.05, rep_len=(300, 6000), rep_copies=(2, 20),
                   rep_div=(0.0, 0.08), n_introns=4000, intron=(50, 2000)),
    # 2 Mb in 4 chromosomes: every-read parity against the oracle.
    "small": dict(chrom_len=[300_000, 500_000, 700_000, 500_000], repeat_share=0.05, rep_len=(200, 2000),
                  rep_copies=(2, 10), rep_div=(0.0, 0.08), n_introns=400, intron=(50, 2000)),
}

#: The paper's simulated read sets: 2M single-end reads of 100 or 250 nt at
#: 0.1% or 1% error; indels are 30% of the errors.  10% of the reads span a
#: splice junction (RNA-seq).
READ_SETS = {
    "T1": dict(lengths=((100, 1.0),), eps=0.001),
    "T2": dict(lengths=((100, 1.0),), eps=0.01),
    "T3": dict(lengths=((250, 1.0),), eps=0.001),
    "T4": dict(lengths=((250, 1.0),), eps=0.01),
}


@dataclass
class Genome:
    """A reference of chromosomes back to back: ``packed`` 2-bit bases,
    ``chrom_offsets`` (n_chrom + 1, in bases), and the planted introns as
    rows (chrom, global start, length, strand: 0 GT..AG, 1 CT..AC)."""
    name: str
    packed: np.ndarray
    chrom_offsets: np.ndarray
    introns: np.ndarray
    _codes: np.ndarray | None = field(default=None, repr=False)

    @property
    def n_bases(self) -> int:
        return int(self.chrom_offsets[-1])

    @property
    def n_chrom(self) -> int:
        return len(self.chrom_offsets) - 1

    def codes(self) -> np.ndarray:
        if self._codes is None:
            self._codes = unpack(self.packed, self.n_bases)
        return self._codes


@dataclass
class ReadSet:
    """Reads (codes, CSR offsets) and where each came from: chromosome,
    forward-strand chromosome position of its first template base, strand,
    and the intron it spans (-1 for none)."""
    name: str
    reads: np.ndarray
    read_offsets: np.ndarray
    chrom: np.ndarray
    pos: np.ndarray
    strand: np.ndarray
    intron: np.ndarray
    _packed: np.ndarray | None = field(default=None, repr=False)

    @property
    def n_reads(self) -> int:
        return len(self.read_offsets) - 1

    def packed_reads(self) -> np.ndarray:
        if self._packed is None:
            self._packed = pack(self.reads)
        return self._packed

    def read(self, r: int) -> np.ndarray:
        return self.reads[self.read_offsets[r]:self.read_offsets[r + 1]]


def _load_genome_fns(lib):
    p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    if not hasattr(lib, "_genome_ready"):
        lib.synth_genome.argtypes = [ctypes.POINTER(GenomeSpec), p, p, p, ctypes.c_int]
        lib.synth_read_lengths.argtypes = [ctypes.POINTER(ReadsSpec), p, ctypes.c_int]
        lib.synth_sample_reads.argtypes = [ctypes.POINTER(ReadsSpec), p, i32, p, p, i64, p, p, p, p, p, p,
                                           ctypes.c_int]
        lib._genome_ready = True
    return lib


def genome(name: str = "small", seed: int = 0, threads: int | None = None, **over) -> Genome:
    """Generate a named reference genome (keyword arguments override the
    recipe: chrom_len, repeat_share, rep_len, rep_copies, rep_div, n_introns,
    intron, margin)."""
    lib = _load_genome_fns(_load())
    g = dict(GENOMES[name], margin=4096)
    g.update(over)
    clen = np.asarray(g["chrom_len"], np.int64)
    off = np.zeros(len(clen) + 1, np.int64)
    np.cumsum(clen, out=off[1:])
    s = GenomeSpec()
    s.seed = seed
    s.n_chrom = len(clen)
    s.repeat_share = g["repeat_share"]
    s.rep_len_min, s.rep_len_max = g["rep_len"]
    s.rep_copies_min, s.rep_copies_max = g["rep_copies"]
    s.rep_div_lo, s.rep_div_hi = g["rep_div"]
    s.n_introns = g["n_introns"]
    s.intron_min, s.intron_max = g["intron"]
    s.margin = g["margin"]
    packed = np.zeros(packed_nbytes(int(off[-1])), np.uint8)
    introns = np.zeros((int(s.n_introns), 4), np.int64)
    rc = lib.synth_genome(ctypes.byref(s), _ptr(off), _ptr(packed), _ptr(introns),
                          threads or min(os.cpu_count() or 1, 32))
    if rc:
        raise RuntimeError(f"synth_genome failed: {rc}")
    return Genome(name, packed, off, introns)


def sample_reads(g: Genome, name: str = "T2", n_reads: int = 2_000_000, seed: int = 1, splice: float = 0.10,
                 indel_share: float = 0.3, min_exon: int = 20, threads: int | None = None, **over) -> ReadSet:
    """Sample a named read set from a genome (keyword arguments override:
    lengths, eps)."""
    lib = _load_genome_fns(_load())
    rs = dict(READ_SETS[name])
    rs.update(over)
    s = ReadsSpec()
    s.seed = seed
    s.n_reads = n_reads
    s.n_len = len(rs["lengths"])
    for k, (v, w) in enumerate(rs["lengths"]):
        s.len_val[k] = v
        s.len_w[k] = w
    s.eps = rs["eps"]
    s.indel_share = indel_share
    s.splice_frac = splice
    s.min_exon = min_exon
    nt = threads or min(os.cpu_count() or 1, 32)
    ln = np.zeros(n_reads, np.int32)
    if lib.synth_read_lengths(ctypes.byref(s), _ptr(ln), nt):
        raise RuntimeError("synth_read_lengths failed")
    roff = np.zeros(n_reads + 1, np.int64)
    np.cumsum(ln, out=roff[1:])
    codes = np.zeros(int(roff[-1]), np.uint8)
    chrom = np.zeros(n_reads, np.int32)
    pos = np.zeros(n_reads, np.int64)
    strand = np.zeros(n_reads, np.int8)
    intron = np.zeros(n_reads, np.int32)
    introns = np.ascontiguousarray(g.introns, np.int64)
    rc = lib.synth_sample_reads(ctypes.byref(s), _ptr(g.chrom_offsets), g.n_chrom, _ptr(g.packed), _ptr(introns),
                                len(introns), _ptr(roff), _ptr(codes), _ptr(chrom), _ptr(pos), _ptr(strand),
                                _ptr(intron), nt)
    if rc:
        raise RuntimeError(f"synth_sample_reads failed: {rc}")
    return ReadSet(name, codes, roff, chrom, pos, strand, intron)
