"""The C-ABI library builds, loads and exports every symbol the headers
under include/ declare (no compute calls: runs without a GPU)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names.update(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_declared_symbols():
    import __graft_entry__
    lib = __graft_entry__._cuda_build_module().build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (sw_\w+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing


def test_binding_covers_declarations_and_loads():
    from paper_1304_0681_gb300 import _swgb
    assert sorted(_swgb.EXPORTS) == _declared()
    assert _swgb.sw_cigar_capacity(100) == 203
    assert _swgb.sw_packed_bytes(0) == 0
    assert _swgb.sw_packed_bytes(1) == 16
    assert _swgb.sw_packed_bytes(64) == 16
    assert _swgb.sw_packed_bytes(65) == 32
    assert _swgb.sw_strerror(-2) == "CIGAR slot too small"
    assert _swgb.sw_plan_rows() == [8, 16, 20, 25, 32, 50]


def test_packing_agrees_with_generator():
    import synth
    from paper_1304_0681_gb300 import _swgb
    for n in (0, 1, 63, 64, 65, 1000, 4097):
        assert synth.packed_nbytes(n) == _swgb.sw_packed_bytes(n)


def test_traceback_mode_setting_is_validated():
    import pytest

    from paper_1304_0681_gb300 import _swgb
    _swgb.sw_set_traceback_mode(_swgb.SW_TB_INT32)
    _swgb.sw_set_traceback_mode(_swgb.SW_TB_AUTO)
    for bad in (-1, 2, 7):
        with pytest.raises(_swgb.SwError):
            _swgb.sw_set_traceback_mode(bad)


def test_seeding_arguments_are_checked_before_any_device_work():
    """Host-side validation of the seeding entry points (no GPU needed)."""
    import ctypes

    from paper_1304_0681_gb300 import _swgb
    lib = _swgb._lib
    assert _swgb.sw_index_table_words(15) == 4 ** 15
    assert _swgb.sw_index_table_words(7) == 0 and _swgb.sw_index_table_words(17) == 0
    bad = [dict(k=7), dict(k=17), dict(min_cal_len=14), dict(stride=0), dict(phase=-1), dict(max_hits=0),
           dict(max_hits=2000), dict(merge_dist=-1), dict(max_window=0), dict(max_window=1 << 21)]
    for kw in bad:
        rc = lib.sw_seed_windows(None, None, None, 1, ctypes.byref(_swgb.SeedParams(**kw)), None, None, 1, None, 0,
                                 None, None)
        assert rc == -1, kw
    # a read of 1,024 bases could keep more hits than the block path holds
    rc = lib.sw_seed_windows(None, None, None, 1, ctypes.byref(_swgb.SeedParams(stride=4, max_hits=200)), None,
                             None, 1, None, 0, None, None)
    assert rc == -5
    assert lib.sw_seed_stats(None, None) == -1


def test_top_hits_arguments_are_checked_before_any_device_work():
    """sw_top_hits: a negative read count or a missing required array is
    SW_ERR_INVALID_ARG; an empty batch succeeds without touching a device."""
    from paper_1304_0681_gb300 import _swgb
    lib = _swgb._lib
    assert lib.sw_top_hits(None, None, -1, None, None, None, None, None, None) == -1
    assert lib.sw_top_hits(None, None, 0, None, None, None, None, None, None) == 0
    for missing in range(3):   # score, cand_offsets, best_score
        args = [1, 1, 5, None, 1, None, None, None, None]
        args[(0, 1, 4)[missing]] = None
        assert lib.sw_top_hits(*args) == -1, missing


def test_filter_entry_points_check_arguments_before_any_device_work():
    """sw_filter_align, sw_filter_select and sw_filter_train_step reject bad
    counts, k outside 1..SW_FILTER_MAX_K, a negative or NaN delta and missing
    arrays before touching a device."""
    import ctypes

    from paper_1304_0681_gb300 import _swgb
    lib = _swgb._lib
    sc = ctypes.byref(_swgb.Scoring(5, -4, -10, -1))
    f = ctypes.c_float

    def rules(*rs):
        arr, n = _swgb._rules(rs)
        return arr, n

    def align(n_reads, n_pairs, k=3, cand=1, model=1, best=1, delta=0.0, rs=None):
        arr, n = rs if rs is not None else rules((1000, k, 0.0, delta))
        return lib.sw_filter_align(1, 1, n_reads, 1, 1, 1, cand, n_pairs, model, arr, n, sc, 1, 1, None,
                                   best, None, None)
    assert align(-1, 0) == -1
    assert align(2, 5, k=0) == -1 and align(2, 5, k=17) == -1
    assert align(2, 5, delta=-0.01) == -1 and align(2, 5, delta=float("nan")) == -1
    assert align(0, 0, delta=0.5) == 0
    assert align(2, 5, rs=rules()) == -1                                  # no rule
    assert align(2, 5, rs=rules((200, 2, 0.0, 0.0), (100, 2, 0.0, 0.0))) == -1   # descending bounds
    assert align(2, 5, rs=rules(*[(i, 1, 0.0, 0.0) for i in range(17)])) == -1   # too many
    assert align(0, 0, rs=rules((100, 2, 0.0, 0.0), (100, 3, 0.0, 0.1))) == 0    # equal bounds are ascending

    def by_length(n_reads, rs, roff=1, pred=1, mask=1):
        arr, n = rs
        return lib.sw_filter_select_by_length(pred, 1, roff, n_reads, arr, n, mask, None)
    two = rules((100, 2, 0.0, 0.0), (200, 3, 0.0, 0.1))
    assert by_length(-1, two) == -1 and by_length(0, two) == 0
    assert by_length(4, two, roff=None) == -1 and by_length(4, two, pred=None) == -1
    assert by_length(4, rules((100, 2, 0.0, -1.0))) == -1 and by_length(4, rules()) == -1

    def select(n_reads, k=3, delta=0.0, pred=1, mask=1):
        return lib.sw_filter_select(pred, 1, n_reads, k, f(0.0), f(delta), mask, None)
    assert select(-1) == -1 and select(4, k=0) == -1 and select(4, k=17) == -1
    assert select(4, delta=-1.0) == -1 and select(4, delta=float("nan")) == -1
    assert select(0) == 0 and select(0, delta=0.25) == 0
    assert select(4, pred=None) == -1 and select(4, mask=None) == -1
    assert align(0, 0) == 0
    assert align(0, 5) == -1
    assert align(3, 5, cand=None) == -1 and align(3, 5, best=None) == -1
    assert align(3, 5, model=None) == -1
    step = lib.sw_filter_train_step
    assert step(1, 1, 1, None, 0, f(1e-3), 1, None) == -1
    assert step(1, 1, 1, None, 8, f(1e-3), 0, None) == -1
    assert step(1, 1, 1, None, 8, f(0.0), 1, None) == -1
    assert step(None, 1, 1, None, 8, f(1e-3), 1, None) == -1


def test_headers_are_plain_c_and_link(tmp_path):
    """Both headers compile as strict C99 with warnings as errors, and a C
    program links against the library and calls its host-only entry points
    (no device needed)."""
    import os

    from paper_1304_0681_gb300 import _swgb
    lib = os.path.abspath(_swgb.LIB_PATH)
    src = tmp_path / "abi_check.c"
    src.write_text(
        '#include "swgb.h"\n#include "swgb_seed.h"\n#include <stdio.h>\n'
        "int main(void) {\n"
        "    sw_scoring_t sc = {5, -4, -10, -1};\n"
        "    sw_seed_params_t sp = {15, 12, 7, 64, 30, 20, 30, 2000, 16384};\n"
        "    (void)sc; (void)sp;\n"
        "    if (sw_cigar_capacity(100) < 203) return 1;\n"
        "    if (sw_index_table_words(15) != (int64_t)1 << 30) return 2;\n"
        "    if (sw_top_hits(0, 0, -1, 0, 0, 0, 0, 0, 0) != SW_ERR_INVALID_ARG) return 3;\n"
        '    printf("%s\\n", sw_strerror(SW_ERR_CAPACITY));\n'
        "    return 0;\n"
        "}\n")
    exe = tmp_path / "abi_check"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src), "-o", str(exe),
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.strip() == _swgb.sw_strerror(-2)
