"""Pins of the CPU oracle against things other than itself.

- brute force: every alignment path of tiny inputs, scored directly
  (sw_brute.c), must reproduce the oracle's H, E and F matrices cell by cell,
  its score and its end cell;
- hand-derived worked examples (tests/golden/sw_worked_examples.txt);
- closed forms on generated sequences (identical strings, one mismatch, a
  1-bp window insertion, a spliced read with a short and a long intron);
- the CIGAR rescored against the strings equals the score;
- invariants: score >= 0, symmetry under swapping read and window, reversal,
  monotonicity in the window;
- the bounded-rectangle traceback equals the full-matrix one.
"""
import numpy as np
import pytest

import oracle
import synth
from sw_checks import encode, load_golden, rescore, decode_ops

SCORINGS = [
    oracle.Scoring(5, -4, -10, -1),
    oracle.Scoring(1, -1, -2, -1),
    oracle.Scoring(2, -3, -5, -2),
    oracle.Scoring(3, 0, -3, -3),
    oracle.Scoring(1, -3, -5, -2),
]


def brute_expect(r, w, sc):
    """H/E/F and (score, end) as their plain definitions give them from the
    exhaustive path tables."""
    bm, bd, bi = oracle.brute_tables(r, w, sc)
    H = np.maximum(np.maximum(bm, bd), np.maximum(bi, 0))
    return H, bd, bi


def first_end(H, score):
    """smallest window index j, then smallest read index i, among H == score"""
    if score == 0:
        return -1, -1
    m1, n1 = H.shape
    for j in range(1, n1):
        for i in range(1, m1):
            if H[i, j] == score:
                return i - 1, j - 1
    raise AssertionError("score not found")


def _brute_case(r, w, sc):
    H, E, F = oracle.matrices(r, w, sc)
    Hb, Eb, Fb = brute_expect(r, w, sc)
    np.testing.assert_array_equal(H[1:, 1:], Hb[1:, 1:])
    np.testing.assert_array_equal(E[1:, 1:], Eb[1:, 1:])
    np.testing.assert_array_equal(F[1:, 1:], Fb[1:, 1:])
    score, ie, je, ops = oracle.align(r, w, sc)
    best = int(Hb[1:, 1:].max()) if Hb[1:, 1:].size else 0
    assert score == max(best, 0)
    assert (ie, je) == first_end(Hb, score)
    if score > 0:
        s2, _, i_end2, _ = rescore(r, w, ops, je, sc)
        assert s2 == score and i_end2 == ie


@pytest.mark.parametrize("alphabet", [2, 4])
def test_brute_force_small(alphabet):
    rng = np.random.default_rng(1000 + alphabet)
    for t in range(3000):
        m, n = rng.integers(1, 6, 2)
        r = rng.integers(0, alphabet, m).astype(np.uint8)
        w = rng.integers(0, alphabet, n).astype(np.uint8)
        _brute_case(r, w, SCORINGS[t % len(SCORINGS)])


def test_brute_force_size7():
    rng = np.random.default_rng(77)
    for t in range(150):
        m, n = rng.integers(5, 8, 2)
        alphabet = 2 if t % 2 else 4
        r = rng.integers(0, alphabet, m).astype(np.uint8)
        w = rng.integers(0, alphabet, n).astype(np.uint8)
        _brute_case(r, w, SCORINGS[t % len(SCORINGS)])


def test_brute_force_edges():
    for sc in SCORINGS:
        for r, w in [("A", "A"), ("A", "C"), ("ACGT", "A"), ("A", "ACGT"), ("AAAA", "AAAA"), ("ACAC", "CACA")]:
            _brute_case(encode(r), encode(w), sc)


@pytest.mark.parametrize("row", load_golden("sw_worked_examples.txt"), ids=lambda r: f"{r['read']}-{r['window']}")
def test_worked_examples(row):
    score, ie, je, ops = oracle.align(encode(row["read"]), encode(row["window"]), oracle.Scoring(*row["scoring"]))
    assert (score, ie, je) == (row["score"], row["i_end"], row["j_end"])
    assert oracle.cigar_string(ops) == row["cigar"]


def _rand(rng, n):
    return rng.integers(0, 4, n).astype(np.uint8)


def test_closed_forms():
    rng = np.random.default_rng(5)
    sc = oracle.DEFAULT_SCORING
    for _ in range(20):
        a = _rand(rng, 100)
        # identical strings: 100 * match, 100M
        assert oracle.align(a, a, sc)[0] == 500
        assert oracle.cigar_string(oracle.align(a, a, sc)[3]) == "100M"
        # one mismatch at 50: 99 * 5 - 4
        b = a.copy()
        b[50] = (b[50] + 1) % 4
        s, ie, je, ops = oracle.align(a, b, sc)
        assert (s, ie, je, oracle.cigar_string(ops)) == (491, 99, 99, "100M")
        # one inserted window base after read base 49, differing from both
        # neighbours so the gap has one placement: 500 - 10, 50M1D50M
        x = next(c for c in range(4) if c != a[49] and c != a[50])
        c = np.concatenate([a[:50], [x], a[50:]]).astype(np.uint8)
        s, ie, je, ops = oracle.align(a, c, sc)
        assert (s, oracle.cigar_string(ops)) == (490, "50M1D50M")
        # read longer than window: window = read[20:70] -> 250, 20S50M30S
        s, ie, je, ops = oracle.align(a, a[20:70], sc)
        assert (s, ie, je, oracle.cigar_string(ops)) == (250, 69, 49, "20S50M30S")


def _spliced_read(rng, intron_len):
    """A read over {A, C, G} and a window holding its halves around an intron
    GT + T...T + AG.  No read base is T, so no read segment matches inside the
    intron; read[48..50] = C, so neither half extends into the intron ends
    (G, T ... A, G) and the gap has a single placement."""
    a = rng.integers(0, 3, 100).astype(np.uint8)
    a[48:51] = 1
    intron = np.full(intron_len, 3, np.uint8)
    intron[0], intron[1] = 2, 3
    intron[-2], intron[-1] = 0, 2
    w = np.concatenate([a[:50], intron, a[50:]]).astype(np.uint8)
    return a, w


def test_spliced_closed_forms():
    rng = np.random.default_rng(9)
    sc = oracle.DEFAULT_SCORING
    for _ in range(5):
        a, w = _spliced_read(rng, 50)
        s, ie, je, ops = oracle.align(a, w, sc)
        # 100 * 5 - 10 - 49 * 1 = 441
        assert (s, ie, je, oracle.cigar_string(ops)) == (441, 99, 149, "50M50D50M")
        a, w = _spliced_read(rng, 1000)
        s, ie, je, ops = oracle.align(a, w, sc)
        # the gap costs more than a half scores: one half, 250; the left half
        # ends at the smaller window index
        assert (s, ie, je, oracle.cigar_string(ops)) == (250, 49, 49, "50M50S")


def test_rescore_and_shape_on_generated():
    wl = synth.generate("parity", seed=3, n_reads=200)
    sc = oracle.DEFAULT_SCORING
    for p in range(wl.n_pairs):
        r = wl.reads[wl.read_offsets[p]:wl.read_offsets[p + 1]]
        w = wl.windows[wl.window_offsets[p]:wl.window_offsets[p + 1]]
        s, ie, je, ops = oracle.align(r, w, sc)
        assert s > 0
        runs = decode_ops(ops)
        core = [x for x in runs if x[1] != "S"]
        assert core[0][1] == "M" and core[-1][1] == "M"
        s2, _, i_end2, _ = rescore(r, w, ops, je, sc)
        assert s2 == s and i_end2 == ie


def test_invariants():
    rng = np.random.default_rng(11)
    for t in range(300):
        sc = SCORINGS[t % len(SCORINGS)]
        m, n = rng.integers(1, 40, 2)
        alphabet = 2 if t % 3 == 0 else 4
        r = rng.integers(0, alphabet, m).astype(np.uint8)
        w = rng.integers(0, alphabet, n).astype(np.uint8)
        s = oracle.align(r, w, sc, cigar=False)[0]
        assert s >= 0
        assert oracle.align(w, r, sc, cigar=False)[0] == s           # symmetric scoring
        assert oracle.align(r[::-1], w[::-1], sc, cigar=False)[0] == s
        ext = np.concatenate([w, rng.integers(0, alphabet, 5).astype(np.uint8)])
        assert oracle.align(r, ext, sc, cigar=False)[0] >= s
        assert oracle.align(r, r, sc, cigar=False)[0] == len(r) * sc.match


def test_rectangle_traceback_equals_full():
    sc_list = SCORINGS
    wl = synth.generate("parity", seed=4, n_reads=150)
    rnd = synth.random_pairs(300, (1, 60), (1, 90), seed=6, alphabet=2)
    for wk in (wl, rnd):
        for p in range(wk.n_pairs):
            sc = sc_list[p % len(sc_list)]
            r = wk.reads[wk.read_offsets[p]:wk.read_offsets[p + 1]]
            w = wk.windows[wk.window_offsets[p]:wk.window_offsets[p + 1]]
            s, ie, je, ops = oracle.align(r, w, sc)
            ops2, jlo = oracle.rect_traceback(r, w, s, ie, je, sc)
            np.testing.assert_array_equal(ops, ops2)


def test_band_traceback_equals_full():
    """Rectangle and band are exactness arguments of the CUDA traceback; the
    oracle checks both against its full matrix on tie-heavy inputs."""
    wl = synth.generate("parity", seed=14, n_reads=150)
    rnd = synth.random_pairs(400, (1, 60), (1, 90), seed=16, alphabet=2)
    spl = synth.generate("uneven", seed=3, n_reads=60)
    for wk in (wl, rnd, spl):
        for p in range(wk.n_pairs):
            sc = SCORINGS[p % len(SCORINGS)]
            r = wk.reads[wk.read_offsets[wk.pair_read[p]]:wk.read_offsets[wk.pair_read[p] + 1]]
            w = wk.windows[wk.window_offsets[p]:wk.window_offsets[p + 1]]
            s, ie, je, ops = oracle.align(r, w, sc)
            np.testing.assert_array_equal(ops, oracle.band_traceback(r, w, s, ie, je, sc))


def test_insertion_bound():
    # 490 with one inserted read base in 101: (5*101 - 10 + 1 - 490) / 6 = 1
    assert oracle.insertion_bound(100, 490) == 1
    assert oracle.insertion_bound(99, 500) == 0


def test_deletion_bound_is_tight_enough():
    # a 1-bp window insertion in an otherwise perfect 100-bp alignment: score
    # 490, so at most (5*100 - 10 - 490) / 1 + 1 = 1 deletion
    assert oracle.deletion_bound(99, 490) == 1
    assert oracle.deletion_bound(99, 500) == 0
    assert oracle.deletion_bound(99, 441) == 50


def test_batch_matches_single():
    wl = synth.generate("parity", seed=2, n_reads=64)
    res = oracle.align_batch(wl.reads, wl.read_offsets, wl.windows, wl.window_offsets, threads=3)
    for p in range(wl.n_pairs):
        r = wl.reads[wl.read_offsets[p]:wl.read_offsets[p + 1]]
        w = wl.windows[wl.window_offsets[p]:wl.window_offsets[p + 1]]
        s, ie, je, ops = oracle.align(r, w)
        o = res["cigar_offsets"][p]
        assert (res["score"][p], res["i_end"][p], res["j_end"][p]) == (s, ie, je)
        np.testing.assert_array_equal(res["ops"][o:o + res["n_ops"][p]], ops)
