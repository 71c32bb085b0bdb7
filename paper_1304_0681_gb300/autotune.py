"""Autotuner for the score kernel's lane plans.

The score pass splits the rows of a read over T lanes holding R rows each.
Which (T, R) is fastest depends on the read-length class (padding, lane
utilisation, register pressure and occupancy), so this module times a set of
candidate plans per class, together with the built-in cost model's plan, on
a sample of the caller's batch with the library's own phase timers, installs
the fastest with sw_set_plan (the cost model's plan unless another beats it
by a margin), and keeps the choice in a small JSON cache keyed by GPU name,
class and scoring.
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


def _admissible(plan, m_max: int, n_max: int, match: int) -> bool:
    """A 16-bit-key class (score bound 511..1022) holds at most 32 rows per
    lane; the library skips overrides with more."""
    bound = match * min(m_max, n_max)
    return plan[1] <= 32 or not 510 < bound <= 1022


def tune(workload, scoring, sample_pairs: int = 400_000, seed: int = 0, use_cache: bool = True,
         keep_margin: float = 0.02) -> dict:
    """Tune every read-length class of a synth.Workload; returns and installs
    {max_read_len: (T, R)}.  The candidates of a class are candidate_plans
    (those its score bound admits) and the built-in cost model's plan, timed
    on up to sample_pairs of the class's pairs; the cost model's plan is kept
    unless another is faster by more than keep_margin."""
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
        n_max = int(n[pairs].max())
        _swgb.sw_set_plan(0, 1, 8)
        model = tuple(_swgb.sw_plan_query(m_max, max(n_max, 1), scoring[0]))
        plans = [model] + [p for p in candidate_plans(m_max) if p != model and _admissible(p, m_max, n_max, scoring[0])]
        times = {}
        for plan in plans:
            try:
                times[plan] = _time_plan(b, scoring, m_max, plan)
            except _swgb.SwError:
                continue
        if times:
            best = min(times, key=times.get)
            if model in times and times[model] <= times[best] * (1.0 + keep_margin):
                best = model
            chosen[m_max] = best
            cache[key] = list(best)
    _swgb.sw_set_plan(0, 1, 8)
    for m_max in sorted(chosen):
        _swgb.sw_set_plan(m_max, *chosen[m_max])
    if use_cache:
        try:
            json.dump(cache, open(CACHE, "w"), indent=1)
        except OSError:
            pass
    return chosen
