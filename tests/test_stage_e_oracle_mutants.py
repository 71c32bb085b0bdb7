"""Each plausible mistake planted in a copy of the Stage E oracle (on the
CPU) must fail at least one of its pins in test_stage_e_oracle.py."""
import importlib.util
import itertools
import sys

import pytest

import test_stage_e_oracle as pins
from oracle import stage_e_oracle

SRC = open(stage_e_oracle.__file__).read()

MUTANTS = {
    # records
    "span_ignores_clip": ("i_start = rr[0][0] if rr and rr[0][1] == OP_S else 0", "i_start = 0"),
    "span_counts_insertions": ("if op in (OP_M, OP_D)", "if op in (OP_M, OP_D, OP_I)"),
    "span_drops_deletions": ("if op in (OP_M, OP_D)", "if op in (OP_M,)"),
    "record_end_off_by_one": ("int(pos) + j_end, i_start", "int(pos) + j_end + 1, i_start"),
    "threshold_strict": ("if score[p] > 0 and score[p] >= min_score:\n            out.append",
                         "if score[p] > 0 and score[p] > min_score:\n            out.append"),
    # junctions
    "minus_marks_swapped": ("if first == (C, T) and last == (A, C):", "if first == (G, T) and last == (A, C):"),
    "plus_end_mark": ("if first == (G, T) and last == (A, G):", "if first == (G, T):"),
    "intron_min_strict": ("if n >= min_intron:", "if n > min_intron:"),
    "intron_end_off_by_one": ("int(pos) + j + n - 1, s", "int(pos) + j + n, s"),
    "deletion_not_advancing": ("                    out.append((int(chrom), int(pos) + j, int(pos) + j + n - 1, s))\n"
                               "            j += n",
                               "                    out.append((int(chrom), int(pos) + j, int(pos) + j + n - 1, s))"),
    "insertions_advance": ("        elif op == OP_M:\n            j += n", "        elif op in (OP_M, OP_I):\n            j += n"),
    # top hits
    "last_on_ties": ("c1 = min(c for s, c in cands if s == s1)", "c1 = max(c for s, c in cands if s == s1)"),
    "second_below_best_only": ("others = [s for s, c in cands if c != c1]", "others = [s for s, c in cands if s < s1]"),
    "second_default_minus_one": ("s2 = max(others) if others else 0", "s2 = max(others) if others else -1"),
    "quality_rounds": ("min(60, (60 * (s1 - s2)) // s1)", "min(60, round(60 * (s1 - s2) / s1))"),
    "quality_scale_100": ("min(60, (60 * (s1 - s2)) // s1)", "min(60, (100 * (s1 - s2)) // s1)"),
    "mask_ignored": ("if mask is None or mask[p]]", "]"),
}


def _mutant(name, tmp_path):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, name
    path = tmp_path / f"stage_e_oracle_{name}.py"
    path.write_text(SRC.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"stage_e_oracle_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


def _pin_calls():
    """Every pin, with each parameter set of its parametrize marks."""
    calls = []
    for n in sorted(dir(pins)):
        f = getattr(pins, n)
        if not (n.startswith("test_") and callable(f)):
            continue
        marks = [m for m in getattr(f, "pytestmark", []) if m.name == "parametrize"]
        if not marks:
            calls.append((n, f, {}))
            continue
        grids = []
        for m in marks:
            names = [s.strip() for s in m.args[0].split(",")] if isinstance(m.args[0], str) else list(m.args[0])
            vals = [v if len(names) > 1 else (v,) for v in m.args[1]]
            grids.append([dict(zip(names, v)) for v in vals])
        for combo in itertools.product(*grids):
            kw = {}
            for d in combo:
                kw.update(d)
            calls.append((n, f, kw))
    return calls


def test_pins_pass_on_the_oracle():
    for n, f, kw in _pin_calls():
        f(**kw)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    mod = _mutant(name, tmp_path)
    monkeypatch.setattr(pins, "se", mod)
    failed = []
    for n, f, kw in _pin_calls():
        try:
            f(**kw)
        except AssertionError:
            failed.append(n)
    assert failed, f"mutant {name} passes every pin"
