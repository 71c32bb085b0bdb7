"""Pins of the learned-filter reference (oracle/filter_oracle.py)."""
import numpy as np

from oracle import filter_oracle as fo
from sw_checks import encode


def test_feature_closed_forms():
    rng = np.random.default_rng(0)
    for _ in range(20):
        m = int(rng.integers(4, 200))
        r = rng.integers(0, 4, m).astype(np.uint8)
        # identical strings: every 4-mer shared, features sum to 1
        assert abs(fo.features(r, r).sum() - 1.0) < 1e-12
        # window holding the read twice: still capped by the read's counts
        assert abs(fo.features(r, np.concatenate([r, r])).sum() - 1.0) < 1e-12
        # disjoint alphabets share nothing
        a = rng.integers(0, 2, m).astype(np.uint8)
        b = (rng.integers(0, 2, m + 5) + 2).astype(np.uint8)
        assert fo.features(a, b).sum() == 0.0
    # homopolymers: A^m against A^n -> only prefix AAA, min(m-3, n-3)/(m-3)
    f = fo.features(np.zeros(10, np.uint8), np.zeros(7, np.uint8))
    assert f[0] == 4 / 7 and f[1:].sum() == 0
    # reads shorter than one 4-mer have no features
    assert fo.features(np.zeros(3, np.uint8), np.zeros(50, np.uint8)).sum() == 0


def test_feature_fold_by_prefix():
    # ACGT and ACGA share prefix ACG (k = 0*16 + 1*4 + 2 = 6)
    r = encode("ACGT")
    w = encode("ACGTACGA")
    f = fo.features(r, w)
    assert f[6] == 1.0 and f.sum() == 1.0
    # a window containing only ACGA shares nothing with a read ACGT
    assert fo.features(encode("ACGT"), encode("ACGA")).sum() == 0.0


def test_kmer_counts_against_string_windows():
    rng = np.random.default_rng(1)
    for _ in range(50):
        s = rng.integers(0, 4, int(rng.integers(0, 40))).astype(np.uint8)
        text = "".join("ACGT"[x] for x in s)
        c = fo.kmer_counts(s)
        for q in range(256):
            kmer = "".join("ACGT"[(q >> sh) & 3] for sh in (6, 4, 2, 0))
            assert c[q] == sum(text[i:i + 4] == kmer for i in range(max(len(text) - 3, 0)))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    P = fo.Params.init(3)
    X = rng.uniform(0, 0.3, (16, fo.N_FEAT))
    t = rng.uniform(0, 1, 16)
    g = fo.backward(P, X, t)
    theta = P.flat()
    assert len(theta) == fo.N_PARAMS == 33153
    idx = rng.choice(len(theta), 300, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num = (fo.loss(fo.Params.from_flat(tp), X, t) - fo.loss(fo.Params.from_flat(tm), X, t)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_forward_closed_forms():
    z = fo.Params(np.zeros((64, 256)), np.zeros(256), np.zeros((256, 64)), np.zeros(64), np.zeros(64), 0.25)
    X = np.random.default_rng(4).uniform(0, 1, (5, 64))
    np.testing.assert_array_equal(fo.forward(z, X)[0], np.full(5, 0.25))
    # a path that copies feature 7 through both ReLUs
    W1 = np.zeros((64, 256)); W1[7, 3] = 1.0
    W2 = np.zeros((256, 64)); W2[3, 5] = 2.0
    w3 = np.zeros(64); w3[5] = 0.5
    P = fo.Params(W1, np.zeros(256), W2, np.zeros(64), w3, 0.0)
    np.testing.assert_allclose(fo.forward(P, X)[0], X[:, 7])
    # negative pre-activations are cut by the ReLU
    P.b1[3] = -10.0
    np.testing.assert_array_equal(fo.forward(P, X)[0], np.zeros(5))
    # the output layer is linear: a negative bias comes through
    n = fo.Params(np.zeros((64, 256)), np.zeros(256), np.zeros((256, 64)), np.zeros(64), np.zeros(64), -0.25)
    np.testing.assert_array_equal(fo.forward(n, X)[0], np.full(5, -0.25))


def test_adam_first_step_is_lr_times_sign():
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = fo.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def _adam_run(grads, lr=0.01):
    th = np.zeros(len(grads[0]))
    m, v = np.zeros_like(th), np.zeros_like(th)
    out = []
    for t, g in enumerate(grads, start=1):
        th, m, v = fo.adam_step(th, np.asarray(g, dtype=np.float64), m, v, t, lr)
        out.append((th.copy(), m.copy(), v.copy()))
    return out


def test_adam_constant_gradient_steps_lr_times_sign():
    """Kingma & Ba (2015), Algorithm 1, with g_t = g for every t: the moment
    recursions sum geometric series, m_t = (1 - b1^t) g and v_t = (1 - b2^t)
    g^2, so the bias-corrected estimates are exactly g and g^2 at every step
    and each step moves theta by lr * g / (|g| + eps) ~ lr * sign(g)."""
    g = np.array([0.5, -2.0, 3.0])
    for t, (th, m, v) in enumerate(_adam_run([g] * 4), start=1):
        np.testing.assert_allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
        np.testing.assert_allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12)
        np.testing.assert_allclose(th, -0.01 * t * np.sign(g), rtol=1e-6)


def test_adam_alternating_gradient_shows_the_carry_over():
    """g, -g, g: by hand from Algorithm 1 (b1 = 0.9, b2 = 0.999).
    Step 2: m_2 = 0.9 * 0.1 g - 0.1 g = -0.01 g, m_2 / (1 - 0.81) = -g / 19;
    v_2 = (1 - b2^2) g^2, so v_2 / (1 - b2^2) = g^2.  The step is -lr * (-g/19)
    / |g| = +lr sign(g) / 19.
    Step 3: m_3 = 0.9 * (-0.01 g) + 0.1 g = 0.091 g, over 1 - 0.729 = 0.271
    gives 91 g / 271; v_3 / (1 - b2^3) = g^2.  The step is -lr * 91/271 sign(g).
    A dropped carry-over (m_t = 0.1 g_t) would give -lr sign(g) * 0.1/0.19 at
    step 2."""
    g = np.array([0.25, -4.0])
    runs = _adam_run([g, -g, g])
    s = np.sign(g)
    np.testing.assert_allclose(runs[0][0], -0.01 * s, rtol=1e-6)
    np.testing.assert_allclose(runs[1][1], -0.01 * g, rtol=1e-12)
    np.testing.assert_allclose(runs[1][0], -0.01 * s + 0.01 * s / 19, rtol=1e-6)
    np.testing.assert_allclose(runs[2][1], 0.091 * g, rtol=1e-12)
    np.testing.assert_allclose(runs[2][0], -0.01 * s + 0.01 * s / 19 - 0.01 * s * 91 / 271, rtol=1e-6)


def test_adam_changing_magnitude():
    """g_1 = 1, g_2 = 3 (one parameter), by hand: m_2 = 0.1 (0.9 * 1 + 3) =
    0.39, bias-corrected 0.39 / 0.19 = 39/19; v_2 = 0.001 (0.999 * 1 + 9) =
    0.009999, bias-corrected 0.009999 / 0.001999 = 9999/1999.  Step 2 moves
    theta by -lr (39/19) / sqrt(9999/1999)."""
    runs = _adam_run([[1.0], [3.0]])
    th2, m2, v2 = runs[1]
    np.testing.assert_allclose(m2, [0.39], rtol=1e-12)
    np.testing.assert_allclose(v2, [0.009999], rtol=1e-12)
    step2 = -0.01 * (39 / 19) / np.sqrt(9999 / 1999)
    np.testing.assert_allclose(th2, [-0.01 + step2], rtol=1e-7)


def test_bf16_round():
    # bf16 keeps 7 fraction bits: next to 1.0 the spacing is 2^-7
    v = np.array([1.0, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -2.5, 3.140625, 1e-40,
                  1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8)])
    r = fo.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                   # a quarter step: down
    assert r[2] == 1.0 + 2 ** -7         # three quarters: up
    assert r[3] == -2.5 and r[4] == 3.140625
    assert r[6] == 1.0                   # exactly halfway: ties to the even neighbour (down)
    assert r[7] == 1.0 + 2 ** -6         # exactly halfway: the even neighbour is above
    assert r[8] == -1.0


def test_select_candidates():
    pred = np.array([0.9, 0.1, 0.5, 0.2, 0.2, 0.8, 0.79, 0.1])
    off = np.array([0, 4, 8])
    sel = fo.select_candidates(pred, off, k=1, tau=0.05)
    # read 0: best 0.9, next 0.5 -> margin 0.4 -> only candidate 0
    # read 1: best 0.8, next 0.79 -> margin 0.01 < tau -> all four
    np.testing.assert_array_equal(sel, [True, False, False, False, True, True, True, True])
    sel = fo.select_candidates(pred, off, k=2, tau=0.0)
    np.testing.assert_array_equal(sel, [True, False, True, False, False, True, True, False])
    best = fo.best_per_read(np.array([5, 9, 1, 2, 7, 3, 8, 0]), off, sel)
    np.testing.assert_array_equal(best, [5, 8])


def test_select_candidates_edges():
    """Exactly k candidates (all kept), a margin equal to tau (only a
    smaller one falls back) and tied predictions (the lower index first);
    predictions exact in fp32."""
    off = np.array([0, 2, 5, 8])
    pred = np.array([0.1, 0.7,            # read 0: two candidates, k = 2
                     0.5, 0.25, 0.0,      # read 1: margin 0.25 between first and second
                     0.5, 0.5, 0.5])      # read 2: three-way tie
    sel = fo.select_candidates(pred, off, k=2, tau=0.0)
    np.testing.assert_array_equal(sel[:2], [True, True])
    np.testing.assert_array_equal(sel[5:], [True, True, False])
    sel = fo.select_candidates(pred, off, k=1, tau=0.25)
    np.testing.assert_array_equal(sel[2:5], [True, False, False])
    np.testing.assert_array_equal(sel[5:], [True, True, True])   # margin 0 < tau: all
    sel = fo.select_candidates(pred, off, k=1, tau=0.0)
    np.testing.assert_array_equal(sel[5:], [True, False, False])


def test_select_candidates_within_delta_of_the_best():
    """The relative rule: beyond the k, a candidate joins when the read's
    best prediction exceeds its own by less than delta (strictly); the
    distance is taken from the best, not from the k-th; a fallback read
    keeps all; delta = 0 adds nothing.  Dyadic predictions, exact in fp32."""
    off = np.array([0, 5, 8, 11])
    pred = np.array([0.875, 0.8125, 0.5, 0.75, 0.84375,   # read 0: best 0.875 at index 0
                     0.5, 0.5, 0.5,                        # read 1: three-way tie
                     0.25, 1.0, 0.9375])                   # read 2: best at index 1
    # read 0, k = 1: 0.875 - 0.84375 = 1/32 < 1/16 joins; 0.875 - 0.8125 = 1/16 does not
    sel = fo.select_candidates(pred, off, k=1, tau=0.0, delta=0.0625)
    np.testing.assert_array_equal(sel[:5], [True, False, False, False, True])
    sel = fo.select_candidates(pred, off, k=1, tau=0.0, delta=0.1)
    np.testing.assert_array_equal(sel[:5], [True, True, False, False, True])
    # k = 2 picks 0.875 and 0.84375; measured from the k-th (0.84375) 0.8125
    # would be 1/32 away and join, measured from the best it is 1/16 away
    sel = fo.select_candidates(pred, off, k=2, tau=0.0, delta=0.0625)
    np.testing.assert_array_equal(sel[:5], [True, False, False, False, True])
    # ties: delta 0 keeps the lower index only, any delta > 0 takes all three
    sel = fo.select_candidates(pred, off, k=1, tau=0.0, delta=0.0)
    np.testing.assert_array_equal(sel[5:8], [True, False, False])
    sel = fo.select_candidates(pred, off, k=1, tau=0.0, delta=2.0 ** -10)
    np.testing.assert_array_equal(sel[5:8], [True, True, True])
    # read 2: 1.0 - 0.9375 = 1/16 < 0.07 joins; 0.25 does not
    sel = fo.select_candidates(pred, off, k=1, tau=0.0, delta=0.07)
    np.testing.assert_array_equal(sel[8:], [False, True, True])
    # a margin below tau falls back to all candidates whatever delta is
    sel = fo.select_candidates(pred, off, k=1, tau=0.05, delta=0.01)
    np.testing.assert_array_equal(sel[:5], [True] * 5)
    # the default adds nothing
    np.testing.assert_array_equal(fo.select_candidates(pred, off, 1, 0.0),
                                  fo.select_candidates(pred, off, 1, 0.0, 0.0))


def test_select_by_length_takes_each_read_s_rule():
    """Per-length rules: a read uses the first rule whose max_read_len is at
    least its length (equality included), a read longer than every bound the
    last rule; the rule's k, tau and delta apply as in select_candidates.
    Dyadic predictions, exact in fp32."""
    pred = np.array([0.875, 0.8125, 0.5, 0.84375,      # read 0 (length 100)
                     0.875, 0.8125, 0.5, 0.84375,      # read 1 (length 101)
                     0.875, 0.8125, 0.5, 0.84375,      # read 2 (length 900)
                     0.5, 0.25, 0.125])                # read 3 (length 150)
    off = np.array([0, 4, 8, 12, 15])
    lengths = np.array([100, 101, 900, 150])
    rules = [(100, 1, 0.0, 0.0), (150, 2, 0.0, 0.0), (400, 1, 0.0, 0.1)]
    assert fo.rule_for_length(rules, 100) == rules[0]
    assert fo.rule_for_length(rules, 101) == rules[1] and fo.rule_for_length(rules, 150) == rules[1]
    assert fo.rule_for_length(rules, 151) == rules[2] and fo.rule_for_length(rules, 10 ** 6) == rules[2]
    sel = fo.select_by_length(pred, off, lengths, rules)
    # read 0: k = 1 -> the best only
    np.testing.assert_array_equal(sel[0:4], [True, False, False, False])
    # read 1: k = 2 -> 0.875 and 0.84375
    np.testing.assert_array_equal(sel[4:8], [True, False, False, True])
    # read 2 (longer than every bound: the last rule): k = 1 plus everything
    # less than 0.1 below 0.875 (0.8125 and 0.84375)
    np.testing.assert_array_equal(sel[8:12], [True, True, False, True])
    # read 3: k = 2 of 3
    np.testing.assert_array_equal(sel[12:15], [True, True, False])
    # one rule reproduces select_candidates
    np.testing.assert_array_equal(fo.select_by_length(pred, off, lengths, [(0, 2, 0.01, 0.05)]),
                                  fo.select_candidates(pred, off, 2, 0.01, 0.05))
