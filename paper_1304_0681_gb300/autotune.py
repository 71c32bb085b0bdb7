"""Autotuner for the score kernel's lane plans.

The score pass splits the rows of a read over T lanes holding R rows each.
Which (T, R) is fastest depends on the read-length class (padding, lane
utilisation, register pressure and occupancy), so this module times a set of
candidate plans per class on a sample of the caller's batch with the
library's own phase timers, installs the fastest with sw_set_plan, and keeps
the choice in a small JSON cache keyed by GPU name and class.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import _swgb
from .device import DeviceBatch, align

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")


def candidate_plans(m_max: int, rows=None):
    """Plans that cover reads up to m_max in one row chunk (or 32 lanes)."""
    rows = rows or _swgb.sw_plan_rows()
    out = []
    for R in rows:
        T = -(-m_max // R)
        if T > 32:
            out.append((32, R))
            continue
        for t in sorted({T, T + 1}):
            if t <= 32 and (t * R - m_max) / max(m_max, 1) <= 0.34:
                out.append((t, R))
    return sorted(set(out))


def _time_plan(batch: DeviceBatch, scoring, m_max: int, plan, reps: int = 3) -> float:
    _swgb.sw_set_plan(0, 1, 8)
    _swgb.sw_set_plan(m_max, *plan)
    align(batch, scoring, cigar=False)
    _swgb.sw_phase_timing(True)
    times = []
    for _ in range(reps):
        align(batch, scoring, cigar=False)
        times.append(_swgb.sw_phase_times()[1])
    _swgb.sw_phase_timing(False)
    return min(times)


def tune(workload, scoring, sample_pairs: int = 200_000, seed: int = 0, use_cache: bool = True) -> dict:
    """Tune every read-length class of a synth.Workload; returns and installs
    {max_read_len: (T, R)}."""
    gpu = torch.cuda.get_device_name()
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except ValueError:
            cache = {}
    m = workload.pair_read_lengths
    n = workload.window_lengths
    # length classes in 16-base steps, as the classifier forms them
    cls = (m + 15) // 16
    chosen = {}
    rng = np.random.default_rng(seed)
    for c in np.unique(cls):
        pairs = np.nonzero(cls == c)[0]
        m_max = int(m[pairs].max())
        key = f"{gpu}|m<={m_max}|n~{int(np.median(n[pairs]))}|{tuple(scoring)}"
        if key in cache:
            chosen[m_max] = tuple(cache[key])
            continue
        pick = np.sort(rng.choice(pairs, min(len(pairs), sample_pairs), replace=False))
        sub = workload.pair_slice(pick)
        b = DeviceBatch.from_packed(sub.packed_reads(), sub.read_offsets, sub.packed_windows(), sub.window_offsets,
                                    cigar=False)
        best = None
        for plan in candidate_plans(m_max):
            try:
                ms = _time_plan(b, scoring, m_max, plan)
            except _swgb.SwError:
                continue
            if best is None or ms < best[0]:
                best = (ms, plan)
        if best is not None:
            chosen[m_max] = best[1]
            cache[key] = list(best[1])
    _swgb.sw_set_plan(0, 1, 8)
    for m_max in sorted(chosen):
        _swgb.sw_set_plan(m_max, *chosen[m_max])
    if use_cache:
        try:
            json.dump(cache, open(CACHE, "w"), indent=1)
        except OSError:
            pass
    return chosen
