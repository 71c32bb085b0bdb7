"""Seeding over the C ABI (include/swgb_seed.h): the k-mer index of a
reference, reads to candidate windows (the paper's Stages C and D and Stage E
tasks i-ii), and the map of a whole batch: seed, extract the windows' bases,
align every read against its windows (Stage E task iii), keep the records
and the best hit per read (task iv).

The kernels do all the work; this module allocates buffers, reads back the
counts that size the next step, and retries once with a larger buffer when
a capacity was too small.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _swgb
from ._swgb import SeedParams, SwError

CAPACITY = -2


def _dev(a, device, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).to(device)


def packed_bytes(n_bases: int) -> int:
    return int(_swgb.sw_packed_bytes(int(n_bases)))


class KmerIndex:
    """The direct-address k-mer index of a packed reference (chromosomes
    back to back, chrom_offsets in bases), built on the device."""

    def __init__(self, packed, chrom_offsets, k: int = 15, device="cuda", stream=None):
        chrom_offsets = np.asarray(chrom_offsets, np.int64)
        self.k = int(k)
        self.n_bases = int(chrom_offsets[-1])
        self.n_chrom = len(chrom_offsets) - 1
        self.chrom_offsets_host = chrom_offsets
        if isinstance(packed, torch.Tensor):
            self.genome = packed.to(device)
        else:
            buf = np.zeros(packed_bytes(self.n_bases), np.uint8)
            buf[:min(len(packed), len(buf))] = np.asarray(packed, np.uint8)[:len(buf)]
            self.genome = _dev(buf, device)
        self.chrom_offsets = _dev(chrom_offsets, device)
        words = _swgb.sw_index_table_words(self.k)
        if words == 0:
            raise ValueError(f"k = {k} outside 8..16")
        self.table = torch.empty(words, dtype=torch.int32, device=device)
        self.positions = torch.empty(max(self.n_bases, 1), dtype=torch.int32, device=device)
        self.n_positions_dev = torch.zeros(1, dtype=torch.int64, device=device)
        _swgb.sw_index_build(self.genome, self.n_bases, self.chrom_offsets, self.n_chrom, self.k, self.table,
                             self.positions, self.n_positions_dev, stream)
        _swgb.sw_sync_status(stream)
        self.n_positions = int(self.n_positions_dev.item())

    def bucket(self, code: int) -> np.ndarray:
        """Positions of k-mer `code` (first base in the low bits), sorted."""
        lo = int(self.table[code - 1].item()) & 0xFFFFFFFF if code else 0
        hi = int(self.table[code].item()) & 0xFFFFFFFF
        return np.sort(self.positions[lo:hi].cpu().numpy().view(np.uint32).astype(np.int64))


_WIN_FIELDS = (("start", torch.int64), ("length", torch.int32), ("chrom", torch.int32), ("pos", torch.int64),
               ("strand", torch.int8), ("pair_read", torch.int64))


def seed_windows(index: KmerIndex, reads, read_offsets, n_reads: int, params: SeedParams | None = None,
                 capacity: int | None = None, stream=None) -> dict:
    """Windows of every read as device tensors (trimmed to the count):
    start, length, chrom, pos, strand, pair_read, cand_offsets, and count."""
    params = params or SeedParams(k=index.k)
    if params.k != index.k:
        raise ValueError("params.k differs from the index's k")
    dev = index.table.device
    cap = int(capacity if capacity is not None else 4 * n_reads + 1024)
    for attempt in range(2):
        out = {n: torch.empty(max(cap, 1), dtype=t, device=dev) for n, t in _WIN_FIELDS}
        out["cand_offsets"] = torch.empty(n_reads + 1, dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        _swgb.sw_seed_windows(index.table, index.positions, index.chrom_offsets, index.n_chrom, params, reads,
                              read_offsets, n_reads, out, cap, cnt, stream)
        try:
            _swgb.sw_sync_status(stream)
        except SwError as e:
            if e.code != CAPACITY or attempt:
                raise
            cap = int(cnt.item())
            continue
        n = int(cnt.item())
        res = {k: v[:n] for k, v in out.items() if k != "cand_offsets"}
        res["cand_offsets"] = out["cand_offsets"]
        res["count"] = n
        return res
    raise AssertionError("unreachable")


def two_strands(reads, read_offsets, n_reads: int, stream=None):
    """(packed reads, offsets) holding each read and then every reverse
    complement: read r's strand s is index r + s * n_reads."""
    total = int(read_offsets[n_reads].item()) if n_reads else 0
    out = torch.zeros(packed_bytes(2 * total), dtype=torch.uint8, device=read_offsets.device)
    off = torch.empty(2 * n_reads + 1, dtype=torch.int64, device=read_offsets.device)
    _swgb.sw_reads_two_strands(reads, read_offsets, n_reads, out, 2 * total, off, stream)
    return out, off


def extract_windows(index: KmerIndex, start, length, n_windows: int, stream=None):
    """(packed window bases, offsets) of the given reference spans."""
    total = int(length[:n_windows].to(torch.int64).sum().item()) if n_windows else 0
    out = torch.empty(packed_bytes(total), dtype=torch.uint8, device=index.genome.device)
    off = torch.empty(n_windows + 1, dtype=torch.int64, device=index.genome.device)
    _swgb.sw_extract_windows(index.genome, index.n_bases, start, length, n_windows, out, total, off, stream)
    return out, off


@dataclass
class Mapped:
    windows: dict          # seed_windows() output
    records_dev: torch.Tensor | None   # sw_record_t rows on the device (min_score given)
    n_records: int
    reads2: torch.Tensor   # both strands of the reads
    reads2_offsets: torch.Tensor
    win_bases: torch.Tensor
    win_offsets: torch.Tensor
    score: torch.Tensor    # per window
    end: torch.Tensor
    cigar: tuple | None
    best_score: torch.Tensor   # per read
    best_cand: torch.Tensor
    second_score: torch.Tensor  # per read: best score of the read's other windows
    mapq: torch.Tensor          # per read: min(60, 60 (best - second) // best)

    def cigar_tuple(self):
        return self.cigar

    @property
    def records(self) -> dict | None:
        """The records as numpy fields (stage_e.records() layout), copied to
        the host on first use."""
        if self.records_dev is None:
            return None
        if not hasattr(self, "_records"):
            from .stage_e import _decode_records
            self._records = _decode_records(self.records_dev, self.n_records)
        return self._records


def map_reads(index: KmerIndex, reads, read_offsets, n_reads: int, scoring, params: SeedParams | None = None,
              cigar: bool = True, stream=None, min_score: int | None = None, junctions=None,
              min_intron: int = 20) -> Mapped:
    """Seed, extract, align every (read strand, window) pair, and pick each
    read's best window (first on ties) with its second-best score and
    mapping quality (sw_top_hits).  With min_score (and a CIGAR), the
    alignments scoring at least min_score also become records in reference
    coordinates, and, given a stage_e.JunctionTable, their deletion runs of
    at least min_intron bases with intron marks are counted in it
    (Stage E, task iv)."""
    win = seed_windows(index, reads, read_offsets, n_reads, params, stream=stream)
    n = win["count"]
    # each call clears the status word the next one reuses: check in between
    reads2, roff2 = two_strands(reads, read_offsets, n_reads, stream)
    _swgb.sw_sync_status(stream)
    wb, woff = extract_windows(index, win["start"], win["length"], n, stream)
    _swgb.sw_sync_status(stream)
    dev = reads.device
    score = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    end = torch.empty(2 * max(n, 1), dtype=torch.int32, device=dev)
    cg = None
    if cigar and n:
        coff = torch.empty(n + 1, dtype=torch.int64, device=dev)
        _swgb.sw_cigar_offsets(roff2, win["pair_read"], n, coff, stream)
        cg = (torch.empty(int(coff[-1].item()), dtype=torch.int32, device=dev), coff,
              torch.empty(n, dtype=torch.int32, device=dev))
    if n:
        _swgb.sw_batch_align_indexed(reads2, roff2, 2 * n_reads, wb, woff, win["pair_read"], n, scoring, score, end,
                                     cg, stream)
        _swgb.sw_sync_status(stream)
    rec_out, n_rec = None, 0
    if min_score is not None and cg is not None and n:
        rec_out = torch.empty((n, 6), dtype=torch.int64, device=dev)
        rec_n = torch.zeros(1, dtype=torch.int64, device=dev)
        _swgb.sw_records(score, end, cg, n, win["chrom"], win["pos"], win["strand"], min_score, rec_out, rec_n, stream)
        _swgb.sw_sync_status(stream)
        n_rec = int(rec_n.item())
        if junctions is not None:
            _swgb.sw_junctions_detect(wb, woff, score, end, cg, n, win["chrom"], win["pos"], min_score, min_intron,
                                      junctions.table, junctions.capacity, stream)
            _swgb.sw_sync_status(stream)
    best, bcand, second, mapq = (torch.empty(max(n_reads, 1), dtype=torch.int32, device=dev) for _ in range(4))
    if n_reads:
        _swgb.sw_top_hits(score, win["cand_offsets"], n_reads, None, best, bcand, second, mapq, stream)
    _swgb.sw_sync_status(stream)
    return Mapped(win, rec_out, n_rec, reads2, roff2, wb, woff, score[:n], end[:2 * n], cg, best[:n_reads],
                  bcand[:n_reads], second[:n_reads], mapq[:n_reads])


@dataclass
class BatchResult:
    best_score: np.ndarray   # per read, -1 when no window
    best_cand: np.ndarray    # index of the best window within the read's windows
    best_start: np.ndarray   # its reference start (-1 when none)
    best_strand: np.ndarray
    mapq: np.ndarray         # mapping quality (sw_top_hits)
    n_windows: int


def _map_host_batch(index: KmerIndex, packed: torch.Tensor, offsets: torch.Tensor, scoring, params, cigar,
                    stream) -> BatchResult:
    dev = index.table.device
    rd = packed.to(dev, non_blocking=True)
    ro = offsets.to(dev, non_blocking=True)
    n_reads = offsets.numel() - 1
    mp = map_reads(index, rd, ro, n_reads, scoring, params, cigar=cigar)
    w = mp.windows
    bc = mp.best_cand.to(torch.int64)
    ok = bc >= 0
    i = torch.where(ok, w["cand_offsets"][:-1] + bc.clamp(min=0), torch.zeros_like(bc))
    if w["count"]:
        start = torch.where(ok, w["start"][i], torch.full_like(bc, -1))
        strand = torch.where(ok, w["strand"][i].to(torch.int64), torch.full_like(bc, -1))
    else:
        start = strand = torch.full_like(bc, -1)
    out = torch.stack([mp.best_score.to(torch.int64), bc, start, strand, mp.mapq.to(torch.int64)]).cpu()
    return BatchResult(out[0].numpy().astype(np.int32), out[1].numpy().astype(np.int32), out[2].numpy(),
                       out[3].numpy().astype(np.int8), out[4].numpy().astype(np.int32), w["count"])


_STREAMS: dict = {}


def _worker_streams(dev, n: int) -> list:
    """The same n worker streams on every call (the library keeps scratch
    per stream: new streams on each call would each grow their own)."""
    key = str(dev)
    pool = _STREAMS.setdefault(key, [])
    while len(pool) < n:
        pool.append(torch.cuda.Stream(device=dev))
    return pool[:n]


def run_on_worker_streams(dev, items: list, fn, n_streams: int = 2) -> list:
    """fn(item, stream) for every item, by n_streams worker threads that each
    drive their own CUDA stream from a pool reused across calls (the library
    keeps separate scratch per stream, so the workers' kernels and host
    round trips overlap).  Returns the results in item order; the first
    exception of any worker is raised after all have stopped."""
    import threading

    results = [None] * len(items)
    errors = []
    next_item = [0]
    lock = threading.Lock()
    streams = _worker_streams(dev, max(n_streams, 1))

    def worker(w):
        torch.cuda.set_device(dev)
        s = streams[w]
        with torch.cuda.stream(s):
            while True:
                with lock:
                    if errors or next_item[0] >= len(items):
                        return
                    k = next_item[0]
                    next_item[0] += 1
                try:
                    results[k] = fn(items[k], s)
                except BaseException as e:  # reported to the caller below
                    with lock:
                        errors.append(e)
                    return

    if n_streams <= 1:
        worker(0)
    else:
        threads = [threading.Thread(target=worker, args=(w,)) for w in range(n_streams)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    if errors:
        raise errors[0]
    return results


def map_batches(index: KmerIndex, batches, scoring, params: SeedParams | None = None, cigar: bool = True,
                n_streams: int = 2) -> list:
    """Map a sequence of host batches, each (packed reads, read offsets) as
    pinned CPU tensors: copy in, seed, extract, align, top hit, copy the
    results back, with n_streams batches in flight on their own streams
    (run_on_worker_streams).  Returns one BatchResult per batch, in order."""
    return run_on_worker_streams(
        index.table.device, list(batches),
        lambda b, s: _map_host_batch(index, b[0], b[1], scoring, params, cigar, s), n_streams)
