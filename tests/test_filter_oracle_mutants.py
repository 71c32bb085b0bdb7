"""Each plausible mistake planted in a copy of the filter oracle (on the
CPU) must fail at least one of its pins in test_filter_oracle.py."""
import importlib.util
import itertools
import sys

import pytest

import test_filter_oracle as pins
from oracle import filter_oracle

SRC = open(filter_oracle.__file__).read()

MUTANTS = {
    # features
    "shared_max": ("shared = np.minimum(", "shared = np.maximum("),
    "fold_by_suffix": ("shared.reshape(N_FEAT, 4).sum(axis=1)", "shared.reshape(4, N_FEAT).sum(axis=0)"),
    "norm_by_m": ("/ float(m - 3)", "/ float(m)"),
    "kmer_first_base_low": ("q = 64 * seq[:-3] + 16 * seq[1:-2] + 4 * seq[2:-1] + seq[3:]",
                            "q = seq[:-3] + 4 * seq[1:-2] + 16 * seq[2:-1] + 64 * seq[3:]"),
    # network
    "no_relu_1": ("a1 = np.maximum(z1, 0.0)", "a1 = z1"),
    "relu_on_output": ("y = a2 @ P.w3 + P.b3", "y = np.maximum(a2 @ P.w3 + P.b3, 0.0)"),
    "grad_without_2": ("dy = 2.0 * (y - t) / B", "dy = (y - t) / B"),
    "grad_no_relu_mask": ("dz2 = da2 * (z2 > 0)", "dz2 = da2"),
    "grad_w1_sign": ("gW1 = X.T @ dz1", "gW1 = -(X.T @ dz1)"),
    # Adam
    "adam_no_bias_correction": ("mh = m / (1 - beta1 ** step)", "mh = m"),
    "adam_no_sqrt": ("np.sqrt(vh) + eps", "vh + eps"),
    "adam_no_momentum_carry": ("m = beta1 * m + (1 - beta1) * grad", "m = (1 - beta1) * grad"),
    "adam_beta1_in_v": ("v = beta2 * v + (1 - beta2) * grad * grad", "v = beta1 * v + (1 - beta2) * grad * grad"),
    "adam_no_v_carry": ("v = beta2 * v + (1 - beta2) * grad * grad", "v = (1 - beta2) * grad * grad"),
    # bf16
    "bf16_truncates": ("u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = u & 0xFFFF0000"),
    "bf16_ties_up": ("u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000", "u = (u + 0x8000) & 0xFFFF0000"),
    # selection and best hit
    "select_all_only_below_k": ("if c <= k:", "if c < k:"),
    "select_ties_high_index": ("np.lexsort((np.arange(c), -pred[a:b]))", "np.lexsort((-np.arange(c), -pred[a:b]))"),
    "select_gap_le": ("if gap < np.float32(tau):", "if gap <= np.float32(tau):"),
    "select_delta_le": ("if top - np.float32(pred[a + j]) < np.float32(delta):",
                        "if top - np.float32(pred[a + j]) <= np.float32(delta):"),
    "select_delta_from_kth": ("top = np.float32(pred[a + order[0]])", "top = np.float32(pred[a + order[k - 1]])"),
    "rule_bound_exclusive": ("        if m <= rule[0]:", "        if m < rule[0]:"),
    "rule_past_bounds_first": ("    return rules[-1]", "    return rules[0]"),
    "select_delta_on_fallback_only": ("        sel[a + order[:k]] = True\n        top",
                                      "        sel[a + order[:k]] = True\n        continue\n        top"),
    "best_is_min": ("out[r] = int(s.max())", "out[r] = int(s.min())"),
}


def _mutant(name, tmp_path):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, name
    path = tmp_path / f"filter_oracle_{name}.py"
    path.write_text(SRC.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"filter_oracle_{name}", path)
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
    monkeypatch.setattr(pins, "fo", mod)
    failed = []
    for n, f, kw in _pin_calls():
        try:
            f(**kw)
        except Exception:  # a pin that fails or crashes on the copy has caught it
            failed.append(n)
    assert failed, f"mutant {name} passes every pin"
