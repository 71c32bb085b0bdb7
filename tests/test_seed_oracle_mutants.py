"""Each plausible mistake planted in a copy of the seeding oracle (on the
CPU) must fail at least one of its pins.  (Dropping the max() when a
region extends a merged one is not a mistake: regions all span k bases and
arrive sorted, so the later end is always the larger.)"""
import importlib.util
import sys

import pytest

import test_seed_oracle as pins
from oracle import seed_oracle

SRC = open(seed_oracle.__file__).read()

MUTANTS = {
    "merge_le": ("a - mb - 1 < p.merge_dist", "a - mb - 1 <= p.merge_dist"),
    "merge_gap": ("a - mb - 1 < p.merge_dist", "a - mb < p.merge_dist"),
    "merge_any_chrom": ("and chrom_of(chrom_offsets, a) == chrom_of(chrom_offsets, ma)", ""),
    "cal_ge": ("b - a + 1 > p.min_cal_len", "b - a + 1 >= p.min_cal_len"),
    "hits_ge": ("len(h) > p.max_hits", "len(h) >= p.max_hits"),
    "no_clamp_left": ("max(a - p.flank, int(chrom_offsets[c]))", "a - p.flank"),
    "no_clamp_right": ("min(b + p.flank, int(chrom_offsets[c + 1]) - 1)", "b + p.flank"),
    "join_le": ("a - jb - 1 < p.max_intron", "a - jb - 1 <= p.max_intron"),
    "join_window": ("max(jb, b) - ja + 1 <= p.max_window", "max(jb, b) - ja <= p.max_window"),
    "one_phase": ("for first in (0, p.phase):", "for first in (0,):"),
    "seed_fit": ("while s + p.k <= m:", "while s + p.k < m:"),
    "no_revcomp": ("for strand, seq in ((0, f), (1, rc)):", "for strand, seq in ((0, f), (1, f[::-1])):"),
}


def _mutant(name, tmp_path):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, name
    path = tmp_path / f"seed_oracle_{name}.py"
    path.write_text(SRC.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"seed_oracle_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod  # dataclasses look their module up
    spec.loader.exec_module(mod)
    mod._lib = seed_oracle._load()
    return mod


def _pin_calls():
    calls = []
    for n in dir(pins):
        f = getattr(pins, n)
        if n.startswith("test_") and callable(f):
            if n == "test_exact_hits_match_naive_search":
                calls += [(n, lambda f=f: f(15))]
            else:
                calls.append((n, f))
    return calls


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    mod = _mutant(name, tmp_path)
    monkeypatch.setattr(pins, "so", mod)
    monkeypatch.setattr(pins, "P", mod.SeedParams())
    failed = []
    for n, f in _pin_calls():
        try:
            f()
        except AssertionError:
            failed.append(n)
    assert failed, f"mutant {name} passes every pin"
