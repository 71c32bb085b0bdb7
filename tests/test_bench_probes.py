"""The bench's roofline probes live in their own library (bench_probes.cu ->
libswgb_probes.so), outside the alignment library: it exports exactly the two
probes, the alignment library exports neither, and invalid arguments are
refused before any device work (no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "libswgb_probes.so")


def _exports(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    return {line.split()[-1] for line in out.splitlines() if " T " in line}


@pytest.fixture(scope="module")
def probes():
    if not os.path.exists(LIB):
        pytest.skip("libswgb_probes.so not built (__graft_entry__.build() builds it)")
    lib = ctypes.CDLL(LIB)
    for fn in (lib.probe_alu, lib.probe_gather):
        fn.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        fn.restype = ctypes.c_int
    return lib


def test_probes_are_not_in_the_alignment_library(probes):
    ours = {s for s in _exports(LIB) if s.startswith("probe_")}
    assert ours == {"probe_alu", "probe_gather"}
    main = _exports(os.path.join(ROOT, "paper_1304_0681_gb300", "libswgb.so"))
    assert not {s for s in main if "probe" in s}


def test_probe_arguments_are_checked(probes):
    out = ctypes.c_double()
    assert probes.probe_alu(7, 10, ctypes.byref(out), None) == -1
    assert probes.probe_alu(-1, 10, ctypes.byref(out), None) == -1
    assert probes.probe_alu(1, 0, ctypes.byref(out), None) == -1
    assert probes.probe_alu(1, 10, None, None) == -1
    assert probes.probe_gather(10, 4, ctypes.byref(out), None) == -1
    assert probes.probe_gather(35, 4, ctypes.byref(out), None) == -1
    assert probes.probe_gather(32, 0, ctypes.byref(out), None) == -1
    assert probes.probe_gather(32, 4, None, None) == -1
