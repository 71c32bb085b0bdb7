"""Autotuner for the score kernel's lane plans.

The score pass splits the rows of a read over T lanes holding R rows each.
Which (T, R) is fastest depends on the read-length class (padding, lane
utilisation, register pressure and occupancy), so this module times a set of
candidate plans of each class on a sample of the caller's whole batch with
the library's own phase timers (one class changed at a time, starting from
the built-in cost model's plans), installs the fastest with sw_set_plan, and
keeps the choice in a small JSON cache keyed by GPU name, classes and
scoring.
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


MAX_CLASSES = 16  # the library holds at most 16 plan overrides


def _install(plans: dict) -> None:
    """One override per class (the classes' longest reads, ascending): each
    class gets exactly its own plan."""
    _swgb.sw_set_plan(0, 1, 8)
    for m_max in sorted(plans):
        _swgb.sw_set_plan(m_max, *plans[m_max])


def _time(batch: DeviceBatch, scoring, reps: int = 3) -> float:
    """Score-pass milliseconds of the batch under the installed plans."""
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


def tune(workload, scoring, sample_pairs: int = 1_000_000, seed: int = 0, use_cache: bool = True,
         keep_margin: float = 0.01) -> dict:
    """Tune every read-length class of a synth.Workload; returns and installs
    {max_read_len: (T, R)}.

    The classes share the GPU in one call (their launches overlap), so a
    plan is timed in the context of the whole batch: on a sample of up to
    sample_pairs pairs of every class, each class in turn tries its
    candidates (candidate_plans that its score bound admits) while every
    other class keeps its current plan, starting from the built-in cost
    model's; a class moves to another plan only when the whole score pass
    gets faster by more than keep_margin.  Batches with more classes than
    the library holds overrides keep the cost model."""
    gpu = torch.cuda.get_device_name()
    m = workload.pair_read_lengths
    n = workload.window_lengths
    # length classes in 16-base steps up to 1,024, as the classifier forms them
    cls = np.where(m <= 1024, (m + 15) // 16, 64 + (m - 1024 + 127) // 128)
    classes = np.unique(cls)
    info = {}
    for c in classes:
        pairs = np.nonzero(cls == c)[0]
        info[int(m[pairs].max())] = int(n[pairs].max())
    _swgb.sw_set_plan(0, 1, 8)
    model = {m_max: tuple(_swgb.sw_plan_query(m_max, max(n_max, 1), scoring[0])) for m_max, n_max in info.items()}
    if len(model) > MAX_CLASSES:
        return {}
    key = f"{gpu}|{sorted(info.items())}|{tuple(scoring)}|{len(m)}"
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except ValueError:
            cache = {}
    if key in cache:
        chosen = {int(k): tuple(v) for k, v in cache[key].items()}
        _install(chosen)
        return chosen
    rng = np.random.default_rng(seed)
    pick = np.arange(len(m)) if len(m) <= sample_pairs else np.sort(rng.choice(len(m), sample_pairs, replace=False))
    sub = workload.pair_slice(pick)
    b = DeviceBatch.from_packed(sub.packed_reads(), sub.read_offsets, sub.packed_windows(), sub.window_offsets,
                                cigar=False)
    chosen = dict(model)
    _install(chosen)
    best_ms = _time(b, scoring)
    for m_max in sorted(info):
        for plan in candidate_plans(m_max):
            if plan == chosen[m_max] or not _admissible(plan, m_max, info[m_max], scoring[0]):
                continue
            trial = dict(chosen)
            trial[m_max] = plan
            try:
                _install(trial)
                ms = _time(b, scoring)
            except _swgb.SwError:
                continue
            if ms < best_ms * (1.0 - keep_margin):
                best_ms, chosen = ms, trial
    _install(chosen)
    if use_cache:
        cache[key] = {str(k): list(v) for k, v in chosen.items()}
        try:
            json.dump(cache, open(CACHE, "w"), indent=1)
        except OSError:
            pass
    return chosen
