"""The pins catch plausible mistakes in the oracle.

Each case copies sw_oracle.c, plants one mistake by text substitution (a
dropped term, a wrong constant, a shifted index, a swapped preference),
compiles the copy on the CPU and runs a reduced set of the pins against it.
Every mutant must fail at least one pin, and the clean copy must pass them
all.  Nothing here touches the CUDA path."""
import os

import numpy as np
import pytest

import oracle
from sw_checks import encode, load_golden, rescore

ORACLE_SRC = os.path.join(os.path.dirname(oracle.__file__), "sw_oracle.c")
BRUTE_SRC = os.path.join(os.path.dirname(oracle.__file__), "sw_brute.c")

MUTANTS = {
    "E opens with extend cost": ("H[i * ld + j - 1] + go, E[i * ld + j - 1] + ge",
                                 "H[i * ld + j - 1] + ge, E[i * ld + j - 1] + ge"),
    "E extends with open cost": ("H[i * ld + j - 1] + go, E[i * ld + j - 1] + ge",
                                 "H[i * ld + j - 1] + go, E[i * ld + j - 1] + go"),
    "F extends with open cost": ("F[(i - 1) * ld + j] + ge", "F[(i - 1) * ld + j] + go"),
    "no zero floor": ("h = max2(h, 0);", "(void)0;"),
    "F term dropped from H": ("h = max2(h, f);", "(void)f;"),
    "match/mismatch swapped": ("const int64_t s = (r[i - 1] == w[j - 1]) ? ma : mi;\n            const int64_t e",
                               "const int64_t s = (r[i - 1] == w[j - 1]) ? mi : ma;\n            const int64_t e"),
    "diagonal index off by one": ("int64_t h = H[(i - 1) * ld + j - 1] + s;", "int64_t h = H[(i - 1) * ld + j] + s;"),
    "end ties to largest j": ("for (int64_t j = 1; j <= n && bj < 0; ++j)", "for (int64_t j = n; j >= 1 && bj < 0; --j)"),
    "end ties to largest i": ("for (int64_t i = 1; i <= m; ++i)\n                if (H[i * (n + 1) + j] == best)",
                              "for (int64_t i = m; i >= 1; --i)\n                if (H[i * (n + 1) + j] == best)"),
    "traceback prefers E over diagonal": (
        "if (h == H[(i - 1) * ld + j - 1] + s) {\n                rev[nrev++] = (uint8_t)OP_M; --i; --j;\n            } else if (h == E[i * ld + j]) {\n                state = 1;",
        "if (h == E[i * ld + j]) {\n                state = 1;\n            } else if (h == H[(i - 1) * ld + j - 1] + s) {\n                rev[nrev++] = (uint8_t)OP_M; --i; --j;"),
    "traceback prefers F over E": ("} else if (h == E[i * ld + j]) {\n                state = 1;\n            } else if (h == F[i * ld + j]) {\n                state = 2;",
                                   "} else if (h == F[i * ld + j]) {\n                state = 2;\n            } else if (h == E[i * ld + j]) {\n                state = 1;"),
    "gap never re-opens in traceback": ("if (E[i * ld + j] == H[i * ld + j - 1] + go) state = 0;",
                                        "if (E[i * ld + j] == H[i * ld + j - 1] + go && j == 1) state = 0;"),
    "trailing clip off by one": ("m - 1 - i_end0", "m - i_end0"),
    "I and D swapped": ("rev[nrev++] = (uint8_t)OP_D;", "rev[nrev++] = (uint8_t)OP_I;"),
    # the bounds behind the rectangle and band tracebacks
    "deletion bound one short": ("return num < 0 ? 0 : num / (-ge) + 1;", "return num < 0 ? 0 : num / (-ge);"),
    "band one diagonal short of the deletions": ("const int64_t dlo = dmax < 0 ? -(i_end + 1) - 1 : dend - dmax;",
                                                 "const int64_t dlo = dmax < 0 ? -(i_end + 1) - 1 : dend - dmax + 1;"),
    "band one diagonal short of the insertions": ("const int64_t dhi = dend + imax;",
                                                  "const int64_t dhi = dend + imax - 1;"),
}


def run_pins(lib) -> list:
    """A reduced pin set; returns the names of the pins that failed."""
    failed = []
    rng = np.random.default_rng(123)
    scorings = [oracle.Scoring(5, -4, -10, -1), oracle.Scoring(2, -3, -5, -2), oracle.Scoring(1, -1, -2, -1)]
    try:
        for t in range(400):
            sc = scorings[t % 3]
            m, n = rng.integers(1, 6, 2)
            a = 2 if t % 2 else 4
            r = rng.integers(0, a, m).astype(np.uint8)
            w = rng.integers(0, a, n).astype(np.uint8)
            H, E, F = oracle.matrices(r, w, sc, lib=lib)
            bm, bd, bi = oracle.brute_tables(r, w, sc)
            Hb = np.maximum(np.maximum(bm, bd), np.maximum(bi, 0))
            if not (np.array_equal(H[1:, 1:], Hb[1:, 1:]) and np.array_equal(E[1:, 1:], bd[1:, 1:])
                    and np.array_equal(F[1:, 1:], bi[1:, 1:])):
                failed.append("brute-matrices")
                break
    except Exception:
        failed.append("brute-matrices(crash)")
    try:
        for row in load_golden("sw_worked_examples.txt"):
            s, ie, je, ops = oracle.align(encode(row["read"]), encode(row["window"]),
                                          oracle.Scoring(*row["scoring"]), lib=lib)
            if (s, ie, je, oracle.cigar_string(ops)) != (row["score"], row["i_end"], row["j_end"], row["cigar"]):
                failed.append("golden")
                break
    except Exception:
        failed.append("golden(crash)")
    try:
        for t in range(200):
            sc = scorings[t % 3]
            r = rng.integers(0, 2, rng.integers(1, 30)).astype(np.uint8)
            w = rng.integers(0, 2, rng.integers(1, 30)).astype(np.uint8)
            s, ie, je, ops = oracle.align(r, w, sc, lib=lib)
            if s > 0:
                s2, _, ie2, _ = rescore(r, w, ops, je, sc)
                if (s2, ie2) != (s, ie):
                    failed.append("rescore")
                    break
    except Exception:
        failed.append("rescore(crash)")
    try:
        # rectangle and band against the full matrix: the golden rows (one
        # of them an exact split read, whose single deletion run makes the
        # deletion bound tight) and tie-heavy random pairs
        cases = [(encode(row["read"]), encode(row["window"]), oracle.Scoring(*row["scoring"]))
                 for row in load_golden("sw_worked_examples.txt")]
        for t in range(150):
            cases.append((rng.integers(0, 2, rng.integers(1, 40)).astype(np.uint8),
                          rng.integers(0, 2, rng.integers(1, 60)).astype(np.uint8), scorings[t % 3]))
        for r, w, sc in cases:
            s, ie, je, ops = oracle.align(r, w, sc, lib=lib)
            if s <= 0:
                continue
            band = oracle.band_traceback(r, w, s, ie, je, sc, lib=lib)
            rect, _ = oracle.rect_traceback(r, w, s, ie, je, sc, lib=lib)
            if not (np.array_equal(band, ops) and np.array_equal(rect, ops)):
                failed.append("band-rectangle")
                break
    except Exception:
        failed.append("band-rectangle(crash)")
    return failed


def _build_variant(tmp_path, name, src_text):
    src = tmp_path / f"{name}.c"
    src.write_text(src_text)
    out = str(tmp_path / f"lib_{name}.so")
    oracle.build(force=True, srcs=[str(src), BRUTE_SRC], out=out)
    return oracle.load_library(out)


def test_clean_copy_passes(tmp_path):
    lib = _build_variant(tmp_path, "clean", open(ORACLE_SRC).read())
    assert run_pins(lib) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    before, after = MUTANTS[name]
    text = open(ORACLE_SRC).read()
    # the recurrence is written out in more than one oracle function: plant
    # the mistake wherever the anchor text occurs
    assert text.count(before) >= 1, f"mutation anchor for {name!r} not found"
    lib = _build_variant(tmp_path, "mut", text.replace(before, after))
    assert run_pins(lib), f"planted mistake {name!r} passed every pin"
