"""GPU parity of the learned candidate filter against oracle/filter_oracle.py.

Tolerances (derived from the arithmetic):
- features: the kernel multiplies the shared count by 1/(m-3) in fp32 and
  rounds to bf16; the oracle divides in fp64 and rounds to bf16.  The fp32
  and fp64 values differ by at most ~1 fp32 ulp, so the bf16 results agree
  except where that ulp crosses a bf16 rounding boundary: at most one bf16
  ulp (2^-8 relative) apart.
- forward: the kernel reads bf16 features and bf16 weights, accumulates in
  fp32 and rounds the 256 first-layer activations to bf16 before layer 2.
  The oracle here does the same roundings in fp64, so what remains is fp32
  accumulation order and activations whose fp32 value sits next to a bf16
  rounding boundary (one bf16 ulp, 2^-8 relative, on a few of 256 terms);
  1e-2 relative plus 1e-3 absolute covers that with margin.
- gradient, fp32 kernel (SW_GRAD_FP32): fp32 forward and backward against
  fp64: relative 1e-3 of the largest gradient component.
- gradient, tensor-core kernel (the default): its products take bf16
  operands (the weights as the serving copies round them, the hidden
  activation, the two error signals).  On inputs built so that every one of
  those roundings and every fp32 sum is exact it must equal the fp64
  gradient up to the final 1/n (2e-6 relative).  On random inputs the
  activation rounding (2^-9 relative per element, through the ReLU masks)
  leaves it within 1e-2 (norm) of the fp64 gradient taken at the bf16
  weights, and within 3e-2 of the exact one.
- Adam: fp32 against fp64, 1e-5 relative.
- selection and best hit: bit-exact (the margin decision is taken in fp32 on
  both sides).
"""
import numpy as np
import pytest

import synth
from oracle import filter_oracle as fo

pytestmark = pytest.mark.gpu
SCORING = (5, -4, -10, -1)


def _batch(wl, cigar=False):
    from paper_1304_0681_gb300 import DeviceBatch
    return DeviceBatch.from_packed(wl.packed_reads(), wl.read_offsets, wl.packed_windows(), wl.window_offsets,
                                   pair_read=wl.pair_read, cigar=cigar)


def _bf16_to_f64(t):
    import torch
    return t.view(torch.bfloat16).float().cpu().numpy().astype(np.float64)


def test_features_match_oracle():
    import torch
    from paper_1304_0681_gb300 import filter as flt
    wl = synth.generate("filter", seed=5, n_reads=120)
    b = _batch(wl)
    co = torch.from_numpy(wl.cand_offsets).cuda()
    got = _bf16_to_f64(flt.features(b, co))
    ref = fo.bf16_round(fo.features_batch(wl.reads, wl.read_offsets, wl.windows, wl.window_offsets, wl.pair_read))
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=2 ** -8, atol=0)
    # edge cases: reads and windows shorter than a 4-mer
    edge = synth.random_pairs(200, (1, 9), (0, 9), seed=7)
    b2 = _batch(edge)
    co2 = torch.arange(edge.n_pairs + 1, dtype=torch.int64, device="cuda")
    got2 = _bf16_to_f64(flt.features(b2, co2))
    ref2 = fo.bf16_round(fo.features_batch(edge.reads, edge.read_offsets, edge.windows, edge.window_offsets,
                                           edge.pair_read))
    np.testing.assert_allclose(got2, ref2, rtol=2 ** -8, atol=0)
    # sequences longer than 258 bases use full-width counters
    long = synth.random_pairs(150, (200, 320), (180, 420), seed=9, alphabet=2)
    b3 = _batch(long)
    co3 = torch.arange(long.n_pairs + 1, dtype=torch.int64, device="cuda")
    got3 = _bf16_to_f64(flt.features(b3, co3))
    ref3 = fo.bf16_round(fo.features_batch(long.reads, long.read_offsets, long.windows, long.window_offsets,
                                           long.pair_read))
    np.testing.assert_allclose(got3, ref3, rtol=2 ** -8, atol=0)


def test_features_of_giant_windows():
    """Windows longer than 65,538 bases, where a 4-mer can occur more often
    than 16-bit counters hold (a homopolymer run here), take 32-bit
    counters; next to them in the same candidate group, ordinary windows."""
    import torch
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(21)
    # 7,997 AAAA in the read, 71,997 in the first window: counted modulo
    # 2^16 the window's would be 6,461 and the shared count would drop
    reads = [np.zeros(8100, np.uint8), rng.integers(0, 4, 300).astype(np.uint8)]
    reads[0][8000:] = rng.integers(0, 4, 100)
    wins = [np.zeros(75_000, np.uint8), rng.integers(0, 4, 500).astype(np.uint8),
            rng.integers(0, 4, 66_000).astype(np.uint8), np.zeros(3, np.uint8),
            rng.integers(0, 4, 1200).astype(np.uint8)]
    wins[0][-3000:] = rng.integers(0, 4, 3000)
    pair_read = np.array([0, 0, 0, 1, 1], np.int64)
    roff = np.concatenate([[0], np.cumsum([len(r) for r in reads])]).astype(np.int64)
    woff = np.concatenate([[0], np.cumsum([len(w) for w in wins])]).astype(np.int64)
    wl = synth.Workload("giant", np.concatenate(reads), roff, np.concatenate(wins), woff, pair_read,
                        np.array([0, 3, 5], np.int64), np.zeros(5, np.uint8), np.zeros(2, np.int32))
    b = _batch(wl)
    co = torch.from_numpy(wl.cand_offsets).cuda()
    got = _bf16_to_f64(flt.features(b, co))
    ref = fo.bf16_round(fo.features_batch(wl.reads, wl.read_offsets, wl.windows, wl.window_offsets, wl.pair_read))
    np.testing.assert_allclose(got, ref, rtol=2 ** -8, atol=0)
    assert ref[0][0] > 0.98  # nearly every read 4-mer is AAAA, all shared


def _model_params(model):
    return fo.Params.from_flat(model.params().cpu().numpy().astype(np.float64))


def test_forward_matches_oracle():
    import torch
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(0)
    model = flt.FilterModel(seed=3)
    n = 1000 + 13  # several 16-row tiles and a ragged tail
    x = rng.uniform(0, 0.4, (n, 64))
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16)
    got = model.forward(xb).cpu().numpy()
    P = _model_params(model)
    Pb = fo.Params(fo.bf16_round(P.W1), P.b1, fo.bf16_round(P.W2), P.b2, P.w3, P.b3)
    X = fo.bf16_round(x)
    a1 = fo.bf16_round(np.maximum(X @ Pb.W1 + Pb.b1, 0))
    ref = np.maximum(a1 @ Pb.W2 + Pb.b2, 0) @ Pb.w3 + Pb.b3
    np.testing.assert_allclose(got, ref, rtol=1e-2, atol=1e-3)


def test_forward_with_many_tiles_per_warp_group():
    """The tensor-memory forward when each of a CTA's two warp groups takes
    several tiles (its mbarrier phases wrap, its tensor-memory columns and
    feature buffer are reused) and the last tile is ragged: every row
    against the oracle on the bf16-rounded network."""
    import torch
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(12)
    model = flt.FilterModel(seed=4)
    n = 152 * 128 * 2 * 3 + 77
    x = rng.uniform(0, 0.4, (n, 64))
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16)
    got = model.forward(xb).cpu().numpy()
    import paper_1304_0681_gb300 as sw
    sw._swgb.sw_sync_status()
    P = _model_params(model)
    Pb = fo.Params(fo.bf16_round(P.W1), P.b1, fo.bf16_round(P.W2), P.b2, P.w3, P.b3)
    X = fo.bf16_round(x)
    a1 = fo.bf16_round(np.maximum(X @ Pb.W1 + Pb.b1, 0))
    ref = np.maximum(a1 @ Pb.W2 + Pb.b2, 0) @ Pb.w3 + Pb.b3
    np.testing.assert_allclose(got, ref, rtol=1e-2, atol=1e-3)


@pytest.fixture
def grad_kernel():
    """Select a gradient kernel for one test, and restore the default."""
    import paper_1304_0681_gb300 as sw
    yield lambda kind: sw._swgb.sw_set_mlp_grad_kernel(kind)
    sw._swgb.sw_set_mlp_grad_kernel(sw._swgb.SW_GRAD_AUTO)


def test_gradient_matches_oracle(grad_kernel):
    import torch
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import filter as flt
    grad_kernel(sw._swgb.SW_GRAD_FP32)
    rng = np.random.default_rng(1)
    model = flt.FilterModel(seed=4)
    n = 300
    x = fo.bf16_round(rng.uniform(0, 0.4, (n, 64)))
    t = rng.uniform(0, 1, n)
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16)
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    idx = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    model.grad(xb, tt, idx)
    got = model.gradient().cpu().numpy().astype(np.float64)
    P = _model_params(model)
    ref = fo.backward(P, x, np.asarray(t, np.float32).astype(np.float64))
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, atol=1e-3 * scale, rtol=0)


def _exact_network(rng):
    """A sparse network whose every bf16 rounding point is exact: weights in
    {+-0.5, +-1} (three per hidden unit in W1, three per output in W2),
    biases and w3 in quarters, so z1, A1, z2, the error signals and dA1 are
    short binary fractions, and fp32 sums of them over tens of thousands of
    samples stay exact."""
    W1 = np.zeros((64, 256))
    for j in range(256):
        W1[rng.choice(64, 3, replace=False), j] = rng.choice([-1.0, -0.5, 0.5, 1.0], 3)
    W2 = np.zeros((256, 64))
    for k in range(64):
        W2[rng.choice(256, 3, replace=False), k] = rng.choice([-1.0, -0.5, 0.5, 1.0], 3)
    b1 = rng.choice([-0.5, 0.0, 0.25, 0.5], 256)
    b2 = rng.choice([-0.25, 0.0, 0.25], 64)
    w3 = rng.choice([-0.5, -0.25, 0.0, 0.25, 0.5], 64)
    return fo.Params(W1, b1, W2, b2, w3, 0.5)


def test_tensor_core_gradient_is_exact_when_every_rounding_is(grad_kernel):
    """The tensor-core kernel on an exactly representable network: features
    in quarters, targets y - delta with delta in {+-0.25, +-0.5, +-1} (the
    output y from the fp64 forward, exact in fp32), so every bf16 operand and
    fp32 sum is exact and the gradient must equal the fp64 one up to the
    final multiplication by 1/n.  20,000 samples in a random order: several
    CTAs that sum more than one 128-sample tile, and a ragged last tile."""
    import torch
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import filter as flt
    grad_kernel(sw._swgb.SW_GRAD_AUTO)
    rng = np.random.default_rng(11)
    P = _exact_network(rng)
    n = 20_000
    x = rng.choice([0.0, 0.25, 0.5, 0.75], (n, 64))
    y, (_, z1, _, z2, _) = fo.forward(P, x)
    assert (z1 > 0).mean() > 0.2 and (z1 <= 0).mean() > 0.2 and (z2 > 0).mean() > 0.2 and (z2 <= 0).mean() > 0.2
    t = y - rng.choice([-1.0, -0.5, -0.25, 0.25, 0.5, 1.0], n)
    model = flt.FilterModel(seed=0)
    model.set_params(P.flat())
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16)
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    assert np.array_equal(tt.cpu().numpy().astype(np.float64), t)
    idx = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    model.grad(xb, tt, idx)
    sw.sw_sync_status()
    got = model.gradient().cpu().numpy().astype(np.float64)
    ref = fo.backward(P, x, t)
    assert np.count_nonzero(ref) > 10_000
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-7 * np.abs(ref).max())


def test_tensor_core_gradient_is_close_to_fp64(grad_kernel):
    """Random network and features: within 1e-2 (norm) of the fp64 gradient
    at the bf16 weights, 3e-2 of the exact gradient; and the same bits on a
    second call (the partial sums are added in a fixed order)."""
    import torch
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import filter as flt
    grad_kernel(sw._swgb.SW_GRAD_AUTO)
    rng = np.random.default_rng(12)
    model = flt.FilterModel(seed=3)
    n = 8192 + 77
    x = fo.bf16_round(rng.uniform(0, 0.5, (n, 64)))
    t = rng.uniform(0, 1, n).astype(np.float32).astype(np.float64)
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16)
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    model.grad(xb, tt)
    g1 = model.gradient().clone()
    model.grad(xb, tt)
    sw.sw_sync_status()
    assert torch.equal(g1, model.gradient())
    got = g1.cpu().numpy().astype(np.float64)
    P = _model_params(model)
    Pb = fo.Params(fo.bf16_round(P.W1), P.b1, fo.bf16_round(P.W2), P.b2, P.w3, P.b3)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(got, fo.backward(Pb, x, t)) < 1e-2
    assert rel(got, fo.backward(P, x, t)) < 3e-2


@pytest.mark.parametrize("kind", ["tensor_core", "fp32"])
def test_gradient_shares_combine_to_the_full_batch(kind, grad_kernel):
    """The data-parallel step: each rank's mean gradient over its share of a
    minibatch, weighted by its share and summed (what the all-reduce does),
    equals the gradient of the whole minibatch; three shares, one empty."""
    import torch
    import paper_1304_0681_gb300 as sw
    from paper_1304_0681_gb300 import filter as flt
    grad_kernel(sw._swgb.SW_GRAD_AUTO if kind == "tensor_core" else sw._swgb.SW_GRAD_FP32)
    rng = np.random.default_rng(6)
    model = flt.FilterModel(seed=7)
    n = 257
    x = fo.bf16_round(rng.uniform(0, 0.4, (n, 64)))
    t = rng.uniform(0, 1, n)
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16)
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    idx = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    model.grad(xb, tt, idx)
    full = model.gradient().clone()
    acc = torch.zeros_like(full)
    for lo, hi in ((0, 100), (100, 100), (100, n)):
        if hi > lo:
            model.grad(xb, tt, idx[lo:hi])
            acc += model.gradient() * ((hi - lo) / n)
    scale = float(full.abs().max())
    np.testing.assert_allclose(acc.cpu().numpy(), full.cpu().numpy(), atol=1e-5 * scale, rtol=0)


def test_adam_matches_oracle():
    import torch
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(2)
    model = flt.FilterModel(seed=5)
    theta0 = model.params().cpu().numpy().astype(np.float64)
    m = np.zeros_like(theta0)
    v = np.zeros_like(theta0)
    th = theta0.copy()
    for step in (1, 2, 3):
        g = rng.normal(0, 1e-2, theta0.shape).astype(np.float32)
        model.gradient().copy_(torch.from_numpy(g))
        model.adam(1e-3)
        th, m, v = fo.adam_step(th, g.astype(np.float64), m, v, step, 1e-3)
    got = model.params().cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, th, rtol=1e-5, atol=1e-7)


def test_select_and_best_match_oracle():
    import torch
    import paper_1304_0681_gb300 as sw
    rng = np.random.default_rng(3)
    counts = rng.integers(1, 40, 500)
    off = np.zeros(501, np.int64)
    np.cumsum(counts, out=off[1:])
    n = int(off[-1])
    pred = np.round(rng.uniform(0, 1, n), 2).astype(np.float32)  # many exact ties
    score = rng.integers(0, 500, n).astype(np.int32)
    dpred, doff = torch.from_numpy(pred).cuda(), torch.from_numpy(off).cuda()
    # delta: the relative rule, with differences of two-decimal predictions
    # landing on the boundary (0.01, 0.05) in fp32 on both sides
    for k, tau, delta in ((1, 0.0, 0.0), (1, 0.05, 0.0), (3, 0.02, 0.0), (8, 0.1, 0.0), (16, 0.0, 0.0),
                          (1, 0.0, 0.01), (1, 0.0, 0.05), (2, 0.01, 0.03), (4, 0.0, 0.12), (3, 0.02, 1.5)):
        mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
        sw._swgb.sw_filter_select(dpred, doff, 500, k, tau, delta, mask)
        ref = fo.select_candidates(pred.astype(np.float64), off, k, tau, delta)
        np.testing.assert_array_equal(mask.cpu().numpy().astype(bool), ref)
        best = torch.zeros(500, dtype=torch.int32, device="cuda")
        cand = torch.zeros(500, dtype=torch.int32, device="cuda")
        sw._swgb.sw_best_per_read(torch.from_numpy(score).cuda(), doff, 500, mask, best, cand)
        np.testing.assert_array_equal(best.cpu().numpy(), fo.best_per_read(score, off, ref))


def test_select_by_length_matches_oracle():
    """sw_filter_select_by_length against the oracle's select_by_length:
    read lengths on and next to every rule bound, reads past the last bound,
    reads without candidates, ties; and its argument checks."""
    import torch
    from paper_1304_0681_gb300 import _swgb
    rng = np.random.default_rng(4)
    nr = 700
    rules = [(100, 1, 0.0, 0.05), (150, 3, 0.02, 0.0), (400, 2, 0.0, 0.12), (800, 4, 0.05, 0.01)]
    lengths = rng.choice([75, 99, 100, 101, 149, 150, 151, 399, 400, 401, 800, 801, 3000], nr)
    counts = rng.integers(0, 30, nr)
    off = np.zeros(nr + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    roff = np.zeros(nr + 1, np.int64)
    np.cumsum(lengths, out=roff[1:])
    n = int(off[-1])
    pred = np.round(rng.uniform(0, 1, n), 2).astype(np.float32)   # exact ties, differences on the bounds
    dpred, doff, droff = (torch.from_numpy(x).cuda() for x in (pred, off, roff))
    for rs in (rules, rules[:1], rules[2:], [(0, 2, 0.0, 0.0), (0, 5, 0.0, 0.3)]):
        mask = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
        _swgb.sw_filter_select_by_length(dpred, doff, droff, nr, rs, mask)
        ref = fo.select_by_length(pred.astype(np.float64), off, lengths, rs)
        np.testing.assert_array_equal(mask.cpu().numpy(), ref.astype(np.uint8), err_msg=str(rs))
    # one rule needs no read offsets
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    _swgb.sw_filter_select_by_length(dpred, doff, None, nr, rules[1:2], mask)
    np.testing.assert_array_equal(mask.cpu().numpy().astype(bool), fo.select_candidates(pred, off, 3, 0.02, 0.0))
    for bad in ([], rules[::-1], [(100, 0, 0.0, 0.0)], [(100, 17, 0.0, 0.0)], [(100, 2, 0.0, -0.5)],
                [(i, 1, 0.0, 0.0) for i in range(17)]):
        with pytest.raises(_swgb.SwError):
            _swgb.sw_filter_select_by_length(dpred, doff, droff, nr, bad, mask)
    with pytest.raises(_swgb.SwError):   # several rules need the read offsets
        _swgb.sw_filter_select_by_length(dpred, doff, None, nr, rules, mask)


def test_masked_alignment():
    import torch
    import paper_1304_0681_gb300 as sw
    from gpu_helpers import oracle_subset
    wl = synth.generate("filter", seed=6, n_reads=60)
    b = _batch(wl)
    rng = np.random.default_rng(4)
    mask = (rng.uniform(0, 1, wl.n_pairs) < 0.3).astype(np.uint8)
    sw._swgb.sw_batch_align_masked(b.reads, b.read_offsets, b.n_reads, b.windows, b.window_offsets, b.pair_read,
                                   torch.from_numpy(mask).cuda(), b.n_pairs, SCORING, b.score, b.end, None)
    sw.sw_sync_status()
    score = b.score.cpu().numpy()
    assert (score[mask == 0] == -1).all()
    sel = np.nonzero(mask)[0]
    ref = oracle_subset(wl, sel, SCORING, cigar=False)
    np.testing.assert_array_equal(score[sel], ref["score"])


def test_training_lowers_loss_and_ranks_true_hits():
    """What the trained network gains over the method without it: against
    the untrained network (same features, same selection) the true candidate
    lands in the top 4 for nearly every read, and the loss drops."""
    import torch
    from paper_1304_0681_gb300 import filter as flt
    wl = synth.generate("filter", seed=8, n_reads=3000)
    b = _batch(wl)
    co = torch.from_numpy(wl.cand_offsets).cuda()
    flt.exhaustive_best(b, co, SCORING)
    feats = flt.features(b, co)
    rl = torch.from_numpy(wl.pair_read_lengths).cuda()
    tgt = flt.targets(b.score, rl, SCORING[0])
    model = flt.FilterModel(seed=1)
    off = wl.cand_offsets

    def top_rank_of_true(pred):
        ranks = []
        for r in range(wl.n_reads):
            p = pred[off[r]:off[r + 1]]
            ranks.append(int(np.sum(p > p[wl.true_cand[r]])))
        return np.array(ranks)

    untrained = top_rank_of_true(model.forward(feats).cpu().numpy())
    before = float(torch.mean((model.forward(feats) - tgt) ** 2))
    losses = model.train(feats, tgt, epochs=10, batch=2048, lr=3e-3)
    assert losses[-1] < 0.5 * before, (before, losses)
    trained = top_rank_of_true(model.forward(feats).cpu().numpy())
    assert np.mean(trained < 4) > 0.97, np.mean(trained < 4)
    assert np.mean(trained < 4) > np.mean(untrained < 4) + 0.3, (np.mean(trained < 4), np.mean(untrained < 4))


def test_tensor_memory_forward_matches_warp_mma():
    """The tcgen05 (tensor-memory) forward and the warp-level MMA forward
    compute the same network: equal up to fp32 summation order, on a batch
    with a ragged last tile; and both match the oracle."""
    import torch
    from paper_1304_0681_gb300 import _swgb
    from paper_1304_0681_gb300 import filter as flt
    rng = np.random.default_rng(9)
    model = flt.FilterModel(seed=6)
    n = 128 * 37 + 55
    x = rng.uniform(0, 0.5, (n, 64))
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16)
    try:
        _swgb.sw_set_mlp_kernel(_swgb.SW_MLP_MMA_SYNC)
        a = model.forward(xb).cpu().numpy()
        _swgb.sw_set_mlp_kernel(_swgb.SW_MLP_AUTO)
        b = model.forward(xb).cpu().numpy()
        _swgb.sw_sync_status()
    finally:
        _swgb.sw_set_mlp_kernel(_swgb.SW_MLP_AUTO)
    np.testing.assert_allclose(b, a, rtol=1e-2, atol=1e-3)
    P = _model_params(model)
    Pb = fo.Params(fo.bf16_round(P.W1), P.b1, fo.bf16_round(P.W2), P.b2, P.w3, P.b3)
    X = fo.bf16_round(x)
    a1 = fo.bf16_round(np.maximum(X @ Pb.W1 + Pb.b1, 0))
    ref = np.maximum(a1 @ Pb.W2 + Pb.b2, 0) @ Pb.w3 + Pb.b3
    np.testing.assert_allclose(b, ref, rtol=1e-2, atol=1e-3)


def test_filter_workload_full_size_sampled():
    """The filter workload at its benchmark size (500k reads, 16.25M
    candidate pairs), scored exhaustively as the benchmark's plain arm does
    (score and end, indexed reads), checked on a sample of pairs."""
    import torch

    import oracle
    from paper_1304_0681_gb300 import filter as flt
    wl = synth.generate("filter", seed=0)
    b = _batch(wl)
    co = torch.from_numpy(wl.cand_offsets).cuda()
    best, cand = flt.exhaustive_best(b, co, SCORING)
    score = b.score.cpu().numpy()
    end = b.end.cpu().numpy().reshape(-1, 2)
    rng = np.random.default_rng(5)
    pairs = np.sort(rng.choice(wl.n_pairs, 2000, replace=False))
    sub = wl.pair_slice(pairs)
    ref = oracle.align_batch(sub.reads, sub.read_offsets, sub.windows, sub.window_offsets,
                             scoring=oracle.Scoring(*SCORING), cigar=False)
    np.testing.assert_array_equal(score[pairs], ref["score"])
    np.testing.assert_array_equal(end[pairs, 0], ref["i_end"])
    np.testing.assert_array_equal(end[pairs, 1], ref["j_end"])
    # the best hit per read is the maximum over its candidates
    reads = rng.choice(wl.n_reads, 500, replace=False)
    bs = best.cpu().numpy()
    for r in reads:
        assert bs[r] == score[wl.cand_offsets[r]:wl.cand_offsets[r + 1]].max()


def test_fullmix_workload_full_size_sampled():
    """The full-mix workload at its full size: 10M reads of 75-800 bases with
    U{1..32} candidates (about 165M pairs), generated on the device.  Both
    benchmark arms run on the whole set: exhaustive SW (score and end) and
    the filtered search (features, network, selection, masked SW; an
    untrained network, so the selection is arbitrary but exercised).  Three
    ranges of reads (first, middle, last), generated on the host, are aligned
    by the oracle: every pair's score and end cell, the best hit per read, and
    the filtered best hit (the maximum over the selected candidates) must
    match."""
    import os

    import torch

    import oracle
    from paper_1304_0681_gb300 import DeviceBatch
    from paper_1304_0681_gb300 import filter as flt
    dw = synth.generate_device("fullmix", seed=0)
    assert dw.n_reads == 10_000_000 and dw.n_pairs > 150_000_000
    n = dw.n_pairs
    b = DeviceBatch(dw.reads, dw.read_offsets, dw.windows, dw.window_offsets, dw.pair_read,
                    torch.zeros(n, dtype=torch.int32, device="cuda"), torch.zeros(2 * n, dtype=torch.int32, device="cuda"),
                    None, None, None)
    best, cand = flt.exhaustive_best(b, dw.cand_offsets, SCORING)
    score = b.score.cpu().numpy()
    end = b.end.cpu().numpy().reshape(-1, 2)
    best = best.cpu().numpy()
    model = flt.FilterModel(seed=3)
    rules = [(112, 4, 0.02, 0.0), (448, 3, 0.02, 0.001), (flt.ALL_LENGTHS, 2, 0.02, 0.0)]
    res = flt.filtered_best(b, dw.cand_offsets, model, rules, SCORING)
    fbest, mask = res.best_score.cpu().numpy(), res.mask.cpu().numpy()
    pred = res.pred.cpu().numpy()
    co = dw.cand_offsets.cpu().numpy()
    span = 1200
    for r0 in (0, dw.n_reads // 2 - span // 2, dw.n_reads - span):
        h = synth.generate("fullmix", seed=0, n_reads=span, first_read=r0)
        p0, p1 = int(co[r0]), int(co[r0 + span])
        np.testing.assert_array_equal(co[r0:r0 + span + 1] - p0, h.cand_offsets)
        sub = h.pair_slice(np.arange(h.n_pairs))
        ref = oracle.align_batch(sub.reads, sub.read_offsets, sub.windows, sub.window_offsets,
                                 scoring=oracle.Scoring(*SCORING), cigar=False, threads=os.cpu_count() or 1)
        np.testing.assert_array_equal(score[p0:p1], ref["score"])
        np.testing.assert_array_equal(end[p0:p1, 0], ref["i_end"])
        np.testing.assert_array_equal(end[p0:p1, 1], ref["j_end"])
        # the selection of these reads, by the rules of their lengths
        np.testing.assert_array_equal(mask[p0:p1] > 0,
                                      fo.select_by_length(pred[p0:p1].astype(np.float64), h.cand_offsets,
                                                          h.read_lengths, rules))
        for r in range(span):
            a, z = h.cand_offsets[r], h.cand_offsets[r + 1]
            assert best[r0 + r] == ref["score"][a:z].max()
            sel = mask[p0 + a:p0 + z] > 0
            assert sel.any() and fbest[r0 + r] == ref["score"][a:z][sel].max()


def test_filtered_batches_pipelined():
    """Host batches of the candidate workload (one of a single read) through
    the filtered search on 1 and 3 worker streams: read for read the top hit,
    its candidate and mapping quality of the single-call search over all
    reads, and the same number of aligned pairs."""
    import torch

    from paper_1304_0681_gb300 import filter as flt
    from paper_1304_0681_gb300 import stage_e
    wl = synth.generate("filter", seed=12, n_reads=1200)
    model = flt.FilterModel(seed=2)   # untrained: an arbitrary but fixed selection
    torch.cuda.synchronize()
    # tau = 0: no margin fallback (an untrained network's predictions lie too
    # close together for any positive margin), so reads with more than k
    # candidates align only k of them
    rules = flt.one_rule(3, 0.0)
    bounds = [0, 300, 301, 700, 1200]
    batches = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        sub = wl.read_slice(a, b)
        batches.append(tuple(torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
                             for x in (sub.packed_reads(), sub.read_offsets, sub.packed_windows(),
                                       sub.window_offsets, sub.pair_read, sub.cand_offsets)))
    whole = _batch(wl)
    co = torch.from_numpy(wl.cand_offsets).cuda()
    res = flt.filtered_best(whole, co, model, rules, SCORING)
    top = stage_e.top_hits(whole.score, co, wl.n_reads, res.mask)
    torch.cuda.synchronize()
    want = {f: top[f].cpu().numpy() for f in ("best_score", "best_cand", "mapq")}
    n_aligned = int(res.mask.sum().item())
    assert 0 < n_aligned < wl.n_pairs
    for ns in (1, 3):
        out = flt.filtered_batches(model, batches, rules, SCORING, n_streams=ns)
        for f in ("best_score", "best_cand", "mapq"):
            np.testing.assert_array_equal(np.concatenate([getattr(o, f) for o in out]), want[f], err_msg=f)
        assert sum(o.aligned_pairs for o in out) == n_aligned


def test_filter_align_in_one_call():
    """sw_filter_align gives the selection, scores, end cells and best hits
    of the step-by-step filtered search (features, network, selection by
    read-length rules, masked SW, best hit), with the caller's mask and with
    the library's; the selection equals the oracle's on the network's own
    predictions."""
    import torch

    from paper_1304_0681_gb300 import _swgb
    from paper_1304_0681_gb300 import filter as flt
    wl = synth.generate("fullmix", seed=14, n_reads=600)
    model = flt.FilterModel(seed=6)
    co = torch.from_numpy(wl.cand_offsets).cuda()
    b = _batch(wl)
    # deltas: quantiles of the distances below each read's best prediction,
    # so that they add candidates beyond the k and leave others out
    pred0 = model.forward(flt.features(b, co)).cpu().numpy()
    counts = np.diff(wl.cand_offsets)
    assert counts.min() >= 1
    top = np.maximum.reduceat(pred0, wl.cand_offsets[:-1])
    gaps = np.repeat(top, counts) - pred0
    rules = [(112, 3, 0.0, float(np.quantile(gaps, 0.3))), (300, 2, 0.0, float(np.quantile(gaps, 0.1))),
             (flt.ALL_LENGTHS, 1, 0.0, 0.0)]
    assert rules[0][3] > 0 and rules[1][3] > 0
    res = flt.filtered_best(b, co, model, rules, SCORING)
    pred = res.pred.cpu().numpy().astype(np.float64)
    ref = fo.select_by_length(pred, wl.cand_offsets, wl.read_lengths, rules)
    np.testing.assert_array_equal(res.mask.cpu().numpy().astype(bool), ref)
    k_of = np.array([fo.rule_for_length(rules, int(m))[1] for m in wl.read_lengths])
    assert ref.sum() > int(np.minimum(counts, k_of).sum())   # delta added candidates
    torch.cuda.synchronize()
    assert 0 < int(res.mask.sum().item()) < wl.n_pairs
    for own_mask in (True, False):
        b2 = _batch(wl)
        mask = torch.full((wl.n_pairs,), 7, dtype=torch.uint8, device="cuda") if own_mask else None
        best = torch.full((wl.n_reads,), -7, dtype=torch.int32, device="cuda")
        cand = torch.full_like(best, -7)
        _swgb.sw_filter_align(b2.reads, b2.read_offsets, wl.n_reads, b2.windows, b2.window_offsets, b2.pair_read, co,
                              wl.n_pairs, model.buf, rules, SCORING, b2.score, b2.end, mask, best, cand)
        _swgb.sw_get_status()
        assert torch.equal(b2.score, b.score) and torch.equal(b2.end, b.end)
        assert torch.equal(best, res.best_score) and torch.equal(cand, res.best_cand)
        if own_mask:
            assert torch.equal(mask, res.mask)
    # no candidates at all: every read gets -1, -1
    zero = torch.zeros(4, dtype=torch.int64, device="cuda")
    best = torch.full((3,), 5, dtype=torch.int32, device="cuda")
    cand = torch.full_like(best, 5)
    _swgb.sw_filter_align(b.reads, b.read_offsets, 3, b.windows, b.window_offsets, b.pair_read, zero, 0, model.buf,
                          rules, SCORING, b.score, b.end, None, best, cand)
    torch.cuda.synchronize()
    assert (best == -1).all() and (cand == -1).all()


def test_filter_train_step_in_one_call():
    """sw_filter_train_step leaves the model buffer (parameters, moments,
    gradient, serving copies) bit for bit as sw_mlp_grad then sw_mlp_adam.
    60 samples fit one block of the gradient kernel, so its float sums run in
    one fixed order (several blocks add their shares with atomics)."""
    import torch

    from paper_1304_0681_gb300 import _swgb
    from paper_1304_0681_gb300 import filter as flt
    wl = synth.generate("filter", seed=15, n_reads=60)
    b = _batch(wl)
    feats = flt.features(b, torch.from_numpy(wl.cand_offsets).cuda())
    tgt = torch.rand(wl.n_pairs, generator=torch.Generator().manual_seed(3)).cuda()
    assert wl.n_pairs >= 180
    idx = torch.arange(0, 180, 3, dtype=torch.int32, device="cuda")
    m1, m2 = flt.FilterModel(seed=9), flt.FilterModel(seed=9)
    for step in (1, 2):
        m1.grad(feats, tgt, idx)
        m1.adam(1e-3)
        _swgb.sw_filter_train_step(m2.buf, feats, tgt, idx, idx.numel(), 1e-3, step)
    torch.cuda.synchronize()
    assert m1.step == 2 and torch.equal(m1.buf, m2.buf)
