"""Learned candidate filter over the C ABI.

The paper aligns each read against every extended CAL.  Here a small network
predicts each candidate's SW score from 4-mer features, only the top-k
candidates of a read (and those predicted within delta of its best) are
aligned, and reads whose top predictions are too close to call (margin below
tau) fall back to aligning every candidate.  (k, tau, delta) may differ by
read length: a selection is a list of rules (max_read_len, k, tau, delta),
the first rule whose bound is at least the read's length applying.
Reported scores are always SW scores of aligned candidates.

Every computation runs in libswgb kernels; this module only allocates the
device buffers and sequences the calls.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _swgb
from .device import DeviceBatch

N_FEAT = 64
ALL_LENGTHS = 2 ** 31 - 1


def one_rule(k: int, tau: float, delta: float = 0.0) -> list:
    """The same (k, tau, delta) for reads of every length."""
    return [(ALL_LENGTHS, int(k), float(tau), float(delta))]


class FilterModel:
    """A model buffer (fp32 parameters, Adam state, gradient, bf16 copies)."""

    def __init__(self, seed: int = 0, device="cuda"):
        self.buf = torch.zeros(_swgb.sw_mlp_bytes() // 4, dtype=torch.float32, device=device)
        self.step = 0
        _swgb.sw_mlp_init(self.buf, seed)

    # parameter views in the documented layout
    def params(self) -> torch.Tensor:
        return self.buf[:33153]

    def set_params(self, flat) -> None:
        self.buf[:33153].copy_(torch.as_tensor(flat, dtype=torch.float32))
        _swgb.sw_mlp_refresh(self.buf)

    def gradient(self) -> torch.Tensor:
        return self.buf[3 * 33153:4 * 33153]

    def forward(self, features: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        n = features.shape[0]
        out = torch.empty(n, dtype=torch.float32, device=features.device) if out is None else out
        _swgb.sw_mlp_forward(self.buf, features, n, out)
        return out

    def grad(self, features, target, idx=None) -> None:
        n = idx.numel() if idx is not None else features.shape[0]
        _swgb.sw_mlp_grad(self.buf, features, target, idx, n)

    def adam(self, lr: float) -> None:
        self.step += 1
        _swgb.sw_mlp_adam(self.buf, lr, self.step)

    def train(self, features: torch.Tensor, target: torch.Tensor, epochs: int = 4, batch: int = 8192,
              lr: float = 2e-3, seed: int = 0, group=None, samples: torch.Tensor | None = None) -> list:
        """Minibatch Adam on the mean squared error; returns the mean loss of
        each epoch measured with the serving forward.  `samples` (int32 row
        indices, repeats allowed) is the multiset an epoch draws from, in a new
        random order each epoch; by default every row once.

        With a process group, every rank holds the same training set and the
        same seed: each takes its share of every minibatch, and the gradients
        are combined by an all-reduce before the (identical) Adam step, so
        all ranks keep the same parameters as one rank training alone."""
        n_rows = features.shape[0]
        gen = torch.Generator(device=features.device)
        gen.manual_seed(seed)
        rank, world = 0, 1
        if group is not None:
            import torch.distributed as dist
            rank, world = dist.get_rank(group), dist.get_world_size(group)
        n = n_rows if samples is None else samples.numel()
        losses = []
        for _ in range(epochs):
            perm = torch.randperm(n, generator=gen, device=features.device)
            perm = (perm if samples is None else samples[perm]).to(torch.int32)
            for s in range(0, n - batch + 1, batch):
                if world == 1:
                    self.grad(features, target, perm[s:s + batch])
                else:
                    lo, hi = minibatch_share(batch, rank, world)
                    if hi > lo:
                        self.grad(features, target, perm[s + lo:s + hi])
                    else:
                        self.gradient().zero_()
                    allreduce_mean_gradient(self.gradient(), hi - lo, batch, group)
                self.adam(lr)
            pred = self.forward(features)
            losses.append(float(torch.mean((pred - target) ** 2)))
        return losses


def minibatch_share(n: int, rank: int, world: int) -> tuple:
    """Rank's contiguous share [lo, hi) of an n-sample minibatch."""
    return n * rank // world, n * (rank + 1) // world


def allreduce_mean_gradient(grad: torch.Tensor, n_local: int, n_total: int, group=None) -> None:
    """In place: a rank's mean gradient over its n_local samples becomes the
    mean over all n_total samples of every rank (weight n_local / n_total,
    then a sum over ranks)."""
    import torch.distributed as dist
    grad.mul_(n_local / n_total)
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)


def features(batch: DeviceBatch, cand_offsets: torch.Tensor) -> torch.Tensor:
    """bf16 features (as int16 storage) of every pair of a read-grouped batch."""
    out = torch.empty((batch.n_pairs, N_FEAT), dtype=torch.int16, device=batch.reads.device)
    _swgb.sw_filter_features(batch.reads, batch.read_offsets, batch.n_reads, batch.windows, batch.window_offsets,
                             cand_offsets, out)
    return out


@dataclass
class FilteredResult:
    best_score: torch.Tensor   # int32 per read
    best_cand: torch.Tensor    # int32 per read (index within the read's candidates)
    mask: torch.Tensor         # uint8 per pair: aligned or not
    pred: torch.Tensor         # float per pair


def filtered_best(batch: DeviceBatch, cand_offsets: torch.Tensor, model: FilterModel, rules, scoring,
                  feats: torch.Tensor | None = None) -> FilteredResult:
    """Features -> network -> selection by the rules (top-k, within delta
    of the best, fallback) -> SW on the selected pairs -> best hit per read
    (score and end only)."""
    feats = features(batch, cand_offsets) if feats is None else feats
    pred = model.forward(feats)
    mask = torch.empty(batch.n_pairs, dtype=torch.uint8, device=pred.device)
    _swgb.sw_filter_select_by_length(pred, cand_offsets, batch.read_offsets, batch.n_reads, rules, mask)
    _swgb.sw_batch_align_masked(batch.reads, batch.read_offsets, batch.n_reads, batch.windows, batch.window_offsets,
                                batch.pair_read, mask, batch.n_pairs, scoring, batch.score, batch.end, None)
    best = torch.empty(batch.n_reads, dtype=torch.int32, device=pred.device)
    cand = torch.empty(batch.n_reads, dtype=torch.int32, device=pred.device)
    _swgb.sw_best_per_read(batch.score, cand_offsets, batch.n_reads, mask, best, cand)
    return FilteredResult(best, cand, mask, pred)


def exhaustive_best(batch: DeviceBatch, cand_offsets: torch.Tensor, scoring):
    """SW on every candidate, best hit per read."""
    _swgb.sw_batch_align_indexed(batch.reads, batch.read_offsets, batch.n_reads, batch.windows, batch.window_offsets,
                                 batch.pair_read, batch.n_pairs, scoring, batch.score, batch.end, None)
    best = torch.empty(batch.n_reads, dtype=torch.int32, device=batch.score.device)
    cand = torch.empty(batch.n_reads, dtype=torch.int32, device=batch.score.device)
    _swgb.sw_best_per_read(batch.score, cand_offsets, batch.n_reads, None, best, cand)
    return best, cand


@dataclass
class FilterBatchResult:
    best_score: np.ndarray   # per read, over the aligned candidates (-1: none)
    best_cand: np.ndarray    # its index within the read's candidates
    mapq: np.ndarray         # mapping quality of the top hit (sw_top_hits)
    aligned_pairs: int


def _filter_host_batch(model: FilterModel, batch, rules, scoring) -> FilterBatchResult:
    """One host batch (packed reads, read offsets, packed windows, window
    offsets, pair -> read, candidate offsets; pinned CPU tensors) through the
    filtered search on the current stream, results copied back."""
    from .stage_e import top_hits
    dev = model.buf.device
    reads, roff, wins, woff, pair_read, coff = (t.to(dev, non_blocking=True) for t in batch)
    n_reads, n_pairs = roff.numel() - 1, woff.numel() - 1
    b = DeviceBatch(reads, roff, wins, woff, pair_read, torch.empty(n_pairs, dtype=torch.int32, device=dev),
                    torch.empty(2 * n_pairs, dtype=torch.int32, device=dev), None, None, None)
    pred = model.forward(features(b, coff))
    mask = torch.empty(n_pairs, dtype=torch.uint8, device=dev)
    _swgb.sw_filter_select_by_length(pred, coff, roff, n_reads, rules, mask)
    _swgb.sw_batch_align_masked(b.reads, b.read_offsets, n_reads, b.windows, b.window_offsets, b.pair_read, mask,
                                n_pairs, scoring, b.score, b.end, None)
    top = top_hits(b.score, coff, n_reads, mask)
    out = torch.cat([top["best_score"], top["best_cand"], top["mapq"],
                     mask.sum(dtype=torch.int64).to(torch.int32).reshape(1)]).cpu().numpy()
    return FilterBatchResult(out[:n_reads], out[n_reads:2 * n_reads], out[2 * n_reads:3 * n_reads],
                             int(out[3 * n_reads]))


def filtered_batches(model: FilterModel, batches, rules, scoring, n_streams: int = 2) -> list:
    """The filtered search over a sequence of host batches (see
    _filter_host_batch for their layout): copy in, features, network,
    selection, SW on the selected pairs, top hits, copy out, with n_streams
    batches in flight on their own streams.  One FilterBatchResult per
    batch, in order."""
    from .seed import run_on_worker_streams
    return run_on_worker_streams(model.buf.device, list(batches),
                                 lambda bt, s: _filter_host_batch(model, bt, rules, scoring), n_streams)


def oversample_top(score: np.ndarray, cand_offsets: np.ndarray, top: int = 1, times: int = 4) -> np.ndarray:
    """Training rows with each read's `top` best-scoring candidates (by SW
    score, ties by index) repeated `times` times and every other candidate
    once: the mean squared error then weighs the ordering at the top of a
    read's list, which decides best-hit recall, above the bulk of decoys.
    Host-side bookkeeping over scores already computed on the GPU."""
    nr = len(cand_offsets) - 1
    counts = np.diff(cand_offsets)
    rid = np.repeat(np.arange(nr), counts)
    order = np.lexsort((np.arange(len(score)), -np.asarray(score), rid))
    rank = np.empty(len(score), np.int64)
    rank[order] = np.arange(len(score)) - np.repeat(cand_offsets[:-1], counts)[order]
    rows = np.arange(len(score), dtype=np.int64)
    return np.concatenate([rows, np.repeat(rows[rank < top], times - 1)]).astype(np.int32)


def targets(score: torch.Tensor, read_len: torch.Tensor, match: int) -> torch.Tensor:
    """Training target of a pair: SW score / (match * read length)."""
    return score.to(torch.float32) / (float(match) * read_len.to(torch.float32))


def _segment_max(vals: np.ndarray, cand_offsets: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """Per read: the largest of its candidates' vals (-1 with no candidates)."""
    out = np.full(len(counts), -1, np.int64)
    nz = counts > 0
    if nz.any():
        out[nz] = np.maximum.reduceat(vals, cand_offsets[:-1][nz])
    return out


def calibrate(pred: np.ndarray, score: np.ndarray, cand_offsets: np.ndarray, recall_target: float,
              ks=(1, 2, 3, 4, 5, 6, 7, 8), taus=None, deltas=None):
    """Pick (k, tau, delta) with the fewest aligned pairs whose best-hit
    recall on a held-out set reaches recall_target; returns (k, tau, delta,
    aligned pairs, recall), or None when no grid point reaches it.  A read
    aligns all its candidates when it has at most k or when its k-th and
    (k+1)-th predictions are closer than tau; otherwise its k best plus
    every candidate predicted within delta of its best (sw_filter_select's
    rule).  Host-side bookkeeping over predictions and exhaustive scores
    already computed on the GPU."""
    taus = taus if taus is not None else [0.0, 0.005, 0.01, 0.02, 0.03, 0.05, 0.08, 0.12, 0.2]
    deltas = deltas if deltas is not None else [0.0, 0.03, 0.05, 0.08, 0.1, 0.12, 0.15, 0.2]
    pred = np.asarray(pred, np.float32)
    score = np.asarray(score, np.int64)
    cand_offsets = np.asarray(cand_offsets, np.int64)
    nr = len(cand_offsets) - 1
    counts = np.diff(cand_offsets)
    rid = np.repeat(np.arange(nr), counts)
    true_best = _segment_max(score, cand_offsets, counts)
    # rank of each candidate within its read by prediction (desc), ties by index
    order = np.lexsort((np.arange(len(pred)), -pred, rid))
    rank = np.empty(len(pred), np.int64)
    rank[order] = np.arange(len(pred)) - np.repeat(cand_offsets[:-1], counts)[order]
    top_pred = np.full(nr, -np.inf, np.float32)
    top_pred[rid[rank == 0]] = pred[rank == 0]
    below_top = top_pred[rid] - pred          # fp32, as the kernel takes it
    best = None
    for k in ks:
        sel_pred = np.full(nr, -np.inf, np.float32)
        nxt_pred = np.full(nr, -np.inf, np.float32)
        m_k = rank == k - 1
        m_k1 = rank == k
        sel_pred[rid[m_k]] = pred[m_k]
        nxt_pred[rid[m_k1]] = pred[m_k1]
        with np.errstate(invalid="ignore"):  # reads with <= k candidates: -inf - -inf
            gap = sel_pred - nxt_pred
        fall_by_tau = [(counts <= k) | (gap < np.float32(tau)) for tau in taus]
        for delta in deltas:
            sel = (rank < k) | (below_top < np.float32(delta))
            kept_best = _segment_max(np.where(sel, score, -1), cand_offsets, counts)
            kept = np.bincount(rid[sel], minlength=nr)
            for tau, fall in zip(taus, fall_by_tau):
                got = np.where(fall, true_best, kept_best)
                recall = float(np.mean(got == true_best))
                aligned = int(np.sum(np.where(fall, counts, kept)))
                if recall >= recall_target and (best is None or aligned < best[3]):
                    best = (k, float(tau), float(delta), aligned, recall)
    return best


# Upper bounds of the read-length classes calibrate_by_length gives rules to
# (about a factor 1.4 apart); longer reads form one more class.
LENGTH_BOUNDS = (80, 112, 160, 224, 320, 448, 640, 896, 1280, 1792, 2560)


def _selection_table(pred, score, cand_offsets, pair_cells, ks, taus, deltas):
    """For every grid point (k, tau, delta): per read whether the selection
    keeps a best-scoring candidate, and the cells and pairs it aligns."""
    nr = len(cand_offsets) - 1
    counts = np.diff(cand_offsets)
    rid = np.repeat(np.arange(nr), counts)
    true_best = _segment_max(score, cand_offsets, counts)
    order = np.lexsort((np.arange(len(pred)), -pred, rid))
    rank = np.empty(len(pred), np.int64)
    rank[order] = np.arange(len(pred)) - np.repeat(cand_offsets[:-1], counts)[order]
    top_pred = np.full(nr, -np.inf, np.float32)
    top_pred[rid[rank == 0]] = pred[rank == 0]
    below_top = top_pred[rid] - pred
    all_cells = np.bincount(rid, weights=pair_cells, minlength=nr)
    for k in ks:
        sel_pred = np.full(nr, -np.inf, np.float32)
        nxt_pred = np.full(nr, -np.inf, np.float32)
        sel_pred[rid[rank == k - 1]] = pred[rank == k - 1]
        nxt_pred[rid[rank == k]] = pred[rank == k]
        with np.errstate(invalid="ignore"):
            gap = sel_pred - nxt_pred
        for delta in deltas:
            kept = (rank < k) | (below_top < np.float32(delta))
            kept_best = _segment_max(np.where(kept, score, -1), cand_offsets, counts)
            kept_cells = np.bincount(rid[kept], weights=pair_cells[kept], minlength=nr)
            kept_pairs = np.bincount(rid[kept], minlength=nr)
            for tau in taus:
                fall = (counts <= k) | (gap < np.float32(tau))
                hit = np.where(fall, true_best, kept_best) == true_best
                yield ((k, float(tau), float(delta)), hit, np.where(fall, all_cells, kept_cells),
                       np.where(fall, counts, kept_pairs))


def calibrate_by_length(pred: np.ndarray, score: np.ndarray, cand_offsets: np.ndarray, read_lengths: np.ndarray,
                        window_lengths: np.ndarray, recall_target: float, bounds=LENGTH_BOUNDS,
                        ks=(1, 2, 3, 4, 5, 6, 7, 8), taus=None, deltas=None):
    """Selection rules by read length: one (k, tau, delta) per length class
    (reads up to each of `bounds`, and longer ones), chosen together so that
    the aligned cells (read length x window length of the selected pairs)
    are fewest while the best-hit recall over all reads reaches
    recall_target.  An exact minimum over the grid: a dynamic program over
    the classes on the number of reads whose best hit is missed.  Returns
    (rules, aligned cells, aligned pairs, recall) or None when no choice
    reaches the target; rules as sw_filter_select_by_length takes them.
    Host-side bookkeeping over predictions and exhaustive scores already
    computed on the GPU."""
    taus = taus if taus is not None else [0.0, 0.01, 0.03]
    deltas = deltas if deltas is not None else [0.0, 0.02, 0.04, 0.06, 0.08, 0.1, 0.12, 0.15, 0.2, 0.25, 0.3]
    pred = np.asarray(pred, np.float32)
    score = np.asarray(score, np.int64)
    cand_offsets = np.asarray(cand_offsets, np.int64)
    read_lengths = np.asarray(read_lengths, np.int64)
    nr = len(cand_offsets) - 1
    if nr == 0:
        return None
    cls = np.searchsorted(np.asarray(bounds), read_lengths, side="left")  # m <= bounds[c]
    n_cls = len(bounds) + 1
    need = int(np.ceil(recall_target * nr - 1e-9))     # reads whose best hit must be kept
    max_miss = nr - need
    if max_miss < 0:
        return None
    pair_cells = (read_lengths[np.repeat(np.arange(nr), np.diff(cand_offsets))] *
                  np.asarray(window_lengths, np.int64)).astype(np.float64)
    # per class and grid point: missed reads, aligned cells, aligned pairs
    opts = {c: [] for c in range(n_cls) if np.any(cls == c)}
    for key, hit, cells_r, pairs_r in _selection_table(pred, score, cand_offsets, pair_cells, ks, taus or [0.0],
                                                       deltas):
        miss = np.bincount(cls[~hit], minlength=n_cls)
        cells = np.bincount(cls, weights=cells_r, minlength=n_cls)
        pairs = np.bincount(cls, weights=pairs_r, minlength=n_cls)
        for c in opts:
            opts[c].append((int(miss[c]), float(cells[c]), int(round(pairs[c])), key))
    # dynamic program: best[b] = fewest cells over the classes so far with b misses
    INF = float("inf")
    best = np.full(max_miss + 1, INF)
    best[0] = 0.0
    picks = []
    for c in sorted(opts):
        nb = np.full(max_miss + 1, INF)
        arg = np.full(max_miss + 1, -1, np.int64)
        for i, (mi, ce, _, _) in enumerate(opts[c]):
            if mi > max_miss:
                continue
            cand = np.full(max_miss + 1, INF)
            cand[mi:] = best[:max_miss + 1 - mi] + ce
            better = cand < nb
            nb[better] = cand[better]
            arg[better] = i
        picks.append((c, arg, best))
        best = nb
    b = int(np.argmin(best))
    if not np.isfinite(best[b]):
        return None
    chosen = {}
    for c, arg, prev in reversed(picks):
        i = int(arg[b])
        chosen[c] = opts[c][i]
        b -= opts[c][i][0]
    rules = []
    for c in sorted(chosen):
        bound = bounds[c] if c < len(bounds) else ALL_LENGTHS
        k, tau, delta = chosen[c][3]
        if rules and rules[-1][1:] == (k, tau, delta):
            rules[-1] = (bound, k, tau, delta)      # the same setting as the class below: one rule
        else:
            rules.append((bound, k, tau, delta))
    rules[-1] = (ALL_LENGTHS,) + rules[-1][1:]
    misses = sum(v[0] for v in chosen.values())
    cells = sum(v[1] for v in chosen.values())
    pairs = sum(v[2] for v in chosen.values())
    return rules, cells, pairs, (nr - misses) / nr
