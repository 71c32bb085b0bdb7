"""Device-resident batches in the layout the C ABI expects.

A DeviceBatch holds the 2-bit packed reads and windows, their int64 offsets,
an optional pair -> read index, and the output buffers (score, end cell and a
CSR CIGAR sized with sw_cigar_capacity) as torch tensors on one CUDA device.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _swgb


def _dev(a, device, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device, non_blocking=False)


@dataclass
class DeviceBatch:
    reads: torch.Tensor            # uint8, packed, 16-byte multiple
    read_offsets: torch.Tensor     # int64, n_reads + 1
    windows: torch.Tensor          # uint8, packed
    window_offsets: torch.Tensor   # int64, n_pairs + 1
    pair_read: torch.Tensor | None  # int64, n_pairs, or None (pair p uses read p)
    score: torch.Tensor            # int32, n_pairs
    end: torch.Tensor              # int32, 2 * n_pairs
    cigar_ops: torch.Tensor | None
    cigar_offsets: torch.Tensor | None
    cigar_n: torch.Tensor | None

    @property
    def n_pairs(self) -> int:
        return self.window_offsets.numel() - 1

    @property
    def n_reads(self) -> int:
        return self.read_offsets.numel() - 1

    @staticmethod
    def from_packed(packed_reads, read_offsets, packed_windows, window_offsets, pair_read=None,
                    cigar: bool = True, device="cuda") -> "DeviceBatch":
        read_offsets = np.asarray(read_offsets, dtype=np.int64)
        window_offsets = np.asarray(window_offsets, dtype=np.int64)
        n_pairs = len(window_offsets) - 1
        for buf, off in ((packed_reads, read_offsets), (packed_windows, window_offsets)):
            need = _swgb.sw_packed_bytes(int(off[-1]))
            if len(buf) < need:
                raise ValueError(f"packed buffer holds {len(buf)} bytes, needs {need}")
        cig_ops = cig_off = cig_n = None
        if cigar:
            rl = np.diff(read_offsets)
            m = rl[np.asarray(pair_read)] if pair_read is not None else rl
            cap = 2 * m.astype(np.int64) + 3
            off = np.zeros(n_pairs + 1, np.int64)
            np.cumsum(cap, out=off[1:])
            cig_off = _dev(off, device)
            cig_ops = torch.zeros(int(off[-1]), dtype=torch.int32, device=device)
            cig_n = torch.zeros(n_pairs, dtype=torch.int32, device=device)
        return DeviceBatch(
            reads=_dev(packed_reads, device), read_offsets=_dev(read_offsets, device),
            windows=_dev(packed_windows, device), window_offsets=_dev(window_offsets, device),
            pair_read=None if pair_read is None else _dev(np.asarray(pair_read, np.int64), device),
            score=torch.zeros(n_pairs, dtype=torch.int32, device=device),
            end=torch.zeros(2 * n_pairs, dtype=torch.int32, device=device),
            cigar_ops=cig_ops, cigar_offsets=cig_off, cigar_n=cig_n)

    def cigar_tuple(self):
        if self.cigar_ops is None:
            return None
        return (self.cigar_ops, self.cigar_offsets, self.cigar_n)


def align(batch: DeviceBatch, scoring, cigar: bool = True, stream=None, sync: bool = True) -> DeviceBatch:
    """Run the batch through sw_batch_align (or its indexed form); with sync,
    wait and raise on device-detected errors."""
    cg = batch.cigar_tuple() if cigar else None
    if batch.pair_read is None:
        _swgb.sw_batch_align(batch.reads, batch.read_offsets, batch.windows, batch.window_offsets, batch.n_pairs,
                             scoring, batch.score, batch.end, cg, stream)
    else:
        _swgb.sw_batch_align_indexed(batch.reads, batch.read_offsets, batch.n_reads, batch.windows,
                                     batch.window_offsets, batch.pair_read, batch.n_pairs, scoring, batch.score,
                                     batch.end, cg, stream)
    if sync:
        _swgb.sw_sync_status(stream)
    return batch


class BatchPlan:
    """A plan for the shape of one DeviceBatch (its offsets and pair map):
    launch decisions and scratch fixed once, so that align() is a fixed
    sequence of launches that a CUDA graph can capture and replay.  The
    batch's bases may change between calls; its offsets must not."""

    def __init__(self, batch: DeviceBatch, scoring, cigar: bool = True, stream=None):
        self.batch = batch
        self.cigar = bool(cigar)
        self.handle = _swgb.sw_plan_create(batch.read_offsets, batch.n_reads, batch.window_offsets,
                                           batch.pair_read, batch.n_pairs, scoring, self.cigar, stream)

    def align(self, stream=None) -> DeviceBatch:
        b = self.batch
        _swgb.sw_plan_align(self.handle, b.reads, b.windows, b.score, b.end,
                            b.cigar_tuple() if self.cigar else None, stream)
        return b

    def status(self, stream=None) -> None:
        _swgb.sw_plan_status(self.handle, stream)

    def close(self) -> None:
        if self.handle:
            _swgb.sw_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
