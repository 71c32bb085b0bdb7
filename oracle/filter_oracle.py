"""Reference of the learned candidate filter -- TEST INFRASTRUCTURE ONLY.

The paper's Stage E aligns every read against all of its extended CALs; the
filter is an addition that ranks the candidates of a read so that only the
best-looking ones get full Smith-Waterman, with exhaustive SW as fallback
and as the reference that best-hit recall is measured against.  This module is the plain fp64
definition the CUDA kernels are checked against; only tests, the smoke check
and the benchmark's CPU leg may use it.

Features (one pair = read r of length m, window w of length n): count the
4-mers of both strings, code q = 64 b0 + 16 b1 + 4 b2 + b3 for bases b0..b3;
per 3-base prefix k = q >> 2 sum the shared counts min(c_r(q), c_w(q)) over
the fourth base, and divide by the read's m - 3 four-mers:

    f[k] = sum_{b} min(c_r(4k + b), c_w(4k + b)) / (m - 3),   k = 0..63

(f = 0 when m < 4).  Network: y = w3 . relu(W2^T relu(W1^T f + b1) + b2) + b3
with W1 64x256, W2 256x64, w3 64; loss = mean (y - t)^2 over the batch,
t = SW score / (match * m).
"""
from __future__ import annotations

import numpy as np

N_FEAT, N_H1, N_H2 = 64, 256, 64


def kmer_counts(seq: np.ndarray) -> np.ndarray:
    """256-bin counts of the 4-mers of a base-code sequence (0..3)."""
    seq = np.asarray(seq, dtype=np.int64)
    c = np.zeros(256, dtype=np.int64)
    if len(seq) >= 4:
        q = 64 * seq[:-3] + 16 * seq[1:-2] + 4 * seq[2:-1] + seq[3:]
        np.add.at(c, q, 1)
    return c


def features(read: np.ndarray, window: np.ndarray) -> np.ndarray:
    """The 64 fp64 features of one (read, window) pair."""
    m = len(read)
    if m < 4:
        return np.zeros(N_FEAT)
    shared = np.minimum(kmer_counts(read), kmer_counts(window))
    return shared.reshape(N_FEAT, 4).sum(axis=1) / float(m - 3)


def features_batch(reads, read_offsets, windows, window_offsets, pair_read) -> np.ndarray:
    n = len(window_offsets) - 1
    out = np.zeros((n, N_FEAT))
    for p in range(n):
        r = int(pair_read[p])
        out[p] = features(reads[read_offsets[r]:read_offsets[r + 1]], windows[window_offsets[p]:window_offsets[p + 1]])
    return out


class Params:
    """fp64 parameters in the layout of the CUDA kernels."""

    def __init__(self, W1, b1, W2, b2, w3, b3):
        self.W1, self.b1, self.W2, self.b2, self.w3 = (np.asarray(a, dtype=np.float64) for a in (W1, b1, W2, b2, w3))
        self.b3 = float(b3)

    @staticmethod
    def init(seed: int = 0) -> "Params":
        """He-scaled uniform initialisation (a fixed, seeded recipe)."""
        rng = np.random.default_rng(seed)
        u = lambda fan_in, shape: rng.uniform(-1, 1, shape) * np.sqrt(6.0 / fan_in)
        return Params(u(N_FEAT, (N_FEAT, N_H1)), np.zeros(N_H1), u(N_H1, (N_H1, N_H2)), np.zeros(N_H2),
                      u(N_H2, (N_H2,)) * 0.1, 0.5)

    def flat(self) -> np.ndarray:
        return np.concatenate([self.W1.ravel(), self.b1, self.W2.ravel(), self.b2, self.w3, [self.b3]])

    @staticmethod
    def from_flat(v) -> "Params":
        v = np.asarray(v, dtype=np.float64)
        sizes = [N_FEAT * N_H1, N_H1, N_H1 * N_H2, N_H2, N_H2, 1]
        parts, o = [], 0
        for s in sizes:
            parts.append(v[o:o + s])
            o += s
        return Params(parts[0].reshape(N_FEAT, N_H1), parts[1], parts[2].reshape(N_H1, N_H2), parts[3], parts[4],
                      parts[5][0])


N_PARAMS = N_FEAT * N_H1 + N_H1 + N_H1 * N_H2 + N_H2 + N_H2 + 1


def forward(P: Params, X: np.ndarray):
    """y and the activations needed by backward."""
    z1 = X @ P.W1 + P.b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ P.W2 + P.b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ P.w3 + P.b3
    return y, (X, z1, a1, z2, a2)


def loss(P: Params, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(P, X)
    return float(np.mean((y - t) ** 2))


def backward(P: Params, X: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Gradient of the mean squared error, flattened like Params.flat()."""
    y, (X, z1, a1, z2, a2) = forward(P, X)
    B = X.shape[0]
    dy = 2.0 * (y - t) / B                    # dL/dy
    gw3 = a2.T @ dy
    gb3 = dy.sum()
    da2 = np.outer(dy, P.w3)
    dz2 = da2 * (z2 > 0)
    gW2 = a1.T @ dz2
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ P.W2.T
    dz1 = da1 * (z1 > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def adam_step(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), fp64; returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round fp32/fp64 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def select_candidates(pred, cand_offsets, k: int, tau: float, delta: float = 0.0):
    """Per read: the k best-predicted candidates, or all of them when the
    gap between the k-th and the (k+1)-th prediction is below tau.  Ties in
    the prediction keep the lower candidate index first.  When the read does
    not fall back, every further candidate predicted within delta of the
    read's best (best - pred < delta) joins the k; delta = 0 adds none.
    Returns a boolean mask over pairs."""
    sel = np.zeros(len(pred), dtype=bool)
    for r in range(len(cand_offsets) - 1):
        a, b = int(cand_offsets[r]), int(cand_offsets[r + 1])
        c = b - a
        if c <= k:
            sel[a:b] = True
            continue
        order = np.lexsort((np.arange(c), -pred[a:b]))
        # the margin decisions are taken in fp32, the precision of the kernel
        gap = np.float32(pred[a + order[k - 1]]) - np.float32(pred[a + order[k]])
        if gap < np.float32(tau):
            sel[a:b] = True
            continue
        sel[a + order[:k]] = True
        top = np.float32(pred[a + order[0]])
        for j in range(c):
            if top - np.float32(pred[a + j]) < np.float32(delta):
                sel[a + j] = True
    return sel


def rule_for_length(rules, m: int):
    """The selection rule of a read of length m: the first of `rules`
    (tuples (max_read_len, k, tau, delta) in ascending max_read_len) with
    m <= max_read_len, else the last one."""
    for rule in rules:
        if m <= rule[0]:
            return rule
    return rules[-1]


def select_by_length(pred, cand_offsets, read_lengths, rules):
    """select_candidates with (k, tau, delta) taken per read from the rule
    of its length (rule_for_length).  Returns a boolean mask over pairs."""
    sel = np.zeros(len(pred), dtype=bool)
    for r in range(len(cand_offsets) - 1):
        a, b = int(cand_offsets[r]), int(cand_offsets[r + 1])
        _, k, tau, delta = rule_for_length(rules, int(read_lengths[r]))
        sel[a:b] = select_candidates(pred[a:b], np.array([0, b - a]), k, tau, delta)
    return sel


def best_per_read(score, cand_offsets, mask=None):
    """Max SW score over the (selected) candidates of each read (-1 if none)."""
    out = np.full(len(cand_offsets) - 1, -1, dtype=np.int64)
    for r in range(len(out)):
        a, b = int(cand_offsets[r]), int(cand_offsets[r + 1])
        s = score[a:b] if mask is None else score[a:b][mask[a:b]]
        if len(s):
            out[r] = int(s.max())
    return out
