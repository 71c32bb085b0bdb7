"""Stage E, task iv over the C ABI: alignment records and splice junctions.

Records are the alignments whose score passes a threshold, with their
reference coordinates; junctions are long deletion runs whose intron starts
and ends with GT ... AG (strand 0) or CT ... AC (strand 1), counted across
batches in a device hash table; top hits are each read's best candidate with
a mapping quality from its best and second-best scores.  The kernels do all the work; this module
allocates buffers and decodes the packed outputs.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _swgb
from .device import DeviceBatch


def records(batch: DeviceBatch, window_chrom, window_pos, window_strand, min_score: int, stream=None) -> dict:
    """Records of a batch already aligned with CIGARs, in pair order:
    numpy arrays pair, ref_start, ref_end, chrom, score, read_start,
    read_end, strand, n_ops."""
    n = batch.n_pairs
    dev = batch.score.device
    out = torch.empty((max(n, 1), 6), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    _swgb.sw_records(batch.score, batch.end, batch.cigar_tuple(), n, window_chrom, window_pos, window_strand,
                     min_score, out, cnt, stream)
    return _decode_records(out, int(cnt.item()))


def top_hits(score: torch.Tensor, cand_offsets: torch.Tensor, n_reads: int, mask: torch.Tensor | None = None,
             stream=None) -> dict:
    """Per read (device int32 tensors): best score, its candidate index,
    second-best score and mapping quality min(60, 60 (S1 - S2) // S1)."""
    dev = score.device
    out = {k: torch.empty(max(n_reads, 1), dtype=torch.int32, device=dev)[:n_reads]
           for k in ("best_score", "best_cand", "second_score", "mapq")}
    _swgb.sw_top_hits(score, cand_offsets, n_reads, mask, out["best_score"], out["best_cand"], out["second_score"],
                      out["mapq"], stream)
    return out


def _decode_records(out: torch.Tensor, k: int) -> dict:
    """numpy fields of the first k sw_record_t rows of a device buffer."""
    a = out[:k].cpu().numpy()
    i32 = a.view(np.int32).reshape(k, 12)
    return {"pair": a[:, 0], "ref_start": a[:, 1], "ref_end": a[:, 2], "chrom": i32[:, 6], "score": i32[:, 7],
            "read_start": i32[:, 8], "read_end": i32[:, 9], "strand": i32[:, 10], "n_ops": i32[:, 11]}


class JunctionTable:
    """A device hash table of splice junctions and their counts (capacity
    slots, a power of two), kept across batches."""

    def __init__(self, capacity: int = 1 << 20, device="cuda"):
        self.capacity = int(capacity)
        self.table = torch.empty(_swgb.sw_junction_table_words(self.capacity), dtype=torch.int64, device=device)
        self.clear()

    def clear(self, stream=None) -> None:
        _swgb.sw_junction_table_clear(self.table, self.capacity, stream)

    def detect(self, batch: DeviceBatch, window_chrom, window_pos, min_score: int, min_intron: int,
               stream=None) -> None:
        _swgb.sw_junctions_detect(batch.windows, batch.window_offsets, batch.score, batch.end, batch.cigar_tuple(),
                                  batch.n_pairs, window_chrom, window_pos, min_score, min_intron, self.table,
                                  self.capacity, stream)

    def export(self, stream=None) -> dict:
        """numpy arrays chrom, start, end, strand, count (slot order)."""
        dev = self.table.device
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        out = torch.empty((self.capacity, 4), dtype=torch.int64, device=dev)
        _swgb.sw_junctions_export(self.table, self.capacity, out, self.capacity, cnt, stream)
        k = min(int(cnt.item()), self.capacity)
        a = out[:k].cpu().numpy()
        i32 = a.view(np.int32).reshape(k, 8)
        return {"start": a[:, 0], "end": a[:, 1], "count": a[:, 2], "chrom": i32[:, 6], "strand": i32[:, 7]}
