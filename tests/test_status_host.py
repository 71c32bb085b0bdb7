"""Host logic of error reporting (no GPU): the device status word that kernels
set with atomicOr maps to the error code a call returns.  In particular a
tensor-core kernel whose bounded mbarrier wait runs out sets the timeout bit,
which must come back as SW_ERR_DEVICE_TIMEOUT (the wait itself is not made to
run out on a GPU: with tensor-core work still in flight that would leave the
kernel's TMEM state undefined).  The mapping is compiled with the host
compiler from the library's own header and checked for every combination of
the five status bits against the documented precedence: invalid input,
unsupported shape, capacity, timeout, internal."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

SRC = r'''
#include <cstdio>
#include "swgb_internal.h"
using namespace swgb;
int main()
{
    printf("%d %d %d %d %d\n", (int)ST_BAD_INPUT, (int)ST_UNSUPPORTED, (int)ST_CAPACITY, (int)ST_TIMEOUT,
           (int)ST_INTERNAL);
    for (int st = 0; st < 32; ++st) printf("%d %d\n", st, status_to_code(st));
    return 0;
}
'''


def _header_codes():
    codes = {}
    with open(os.path.join(ROOT, "include", "swgb.h")) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and parts[0] == "#define" and parts[1].startswith("SW_ERR_"):
                codes[parts[1]] = int(parts[2].split("/")[0].strip("()"))
    return codes


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and CUDA headers")
def test_status_bits_map_to_error_codes(tmp_path):
    hdr = _header_codes()
    SW_OK = 0
    SW_ERR_INTERNAL, SW_ERR_CAPACITY = hdr["SW_ERR_INTERNAL"], hdr["SW_ERR_CAPACITY"]
    SW_ERR_DEVICE_TIMEOUT, SW_ERR_UNSUPPORTED = hdr["SW_ERR_DEVICE_TIMEOUT"], hdr["SW_ERR_UNSUPPORTED"]
    SW_ERR_DEVICE_INPUT = hdr["SW_ERR_DEVICE_INPUT"]
    assert len({SW_OK, SW_ERR_INTERNAL, SW_ERR_CAPACITY, SW_ERR_DEVICE_TIMEOUT, SW_ERR_UNSUPPORTED,
                SW_ERR_DEVICE_INPUT}) == 6
    src = tmp_path / "status_check.cpp"
    src.write_text(SRC)
    exe = tmp_path / "status_check"
    inc = os.path.join(ROOT, "paper_1304_0681_gb300", "csrc")
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    bad, unsup, cap, timeout, internal = map(int, out[0].split())
    # five distinct single bits
    assert sorted([bad, unsup, cap, timeout, internal]) == [1, 2, 4, 8, 16]
    got = dict(tuple(map(int, line.split())) for line in out[1:] if line.strip())
    assert len(got) == 32
    for st, code in got.items():
        if st & bad:
            want = SW_ERR_DEVICE_INPUT
        elif st & unsup:
            want = SW_ERR_UNSUPPORTED
        elif st & cap:
            want = SW_ERR_CAPACITY
        elif st & timeout:
            want = SW_ERR_DEVICE_TIMEOUT
        elif st & internal:
            want = SW_ERR_INTERNAL
        else:
            want = SW_OK
        assert code == want, (st, code, want)
    # the timeout bit alone, and with the internal bit, is a timeout
    assert got[timeout] == SW_ERR_DEVICE_TIMEOUT
    assert got[timeout | internal] == SW_ERR_DEVICE_TIMEOUT


def test_timeout_has_a_message():
    """sw_strerror names the timeout (host-only call of the built library)."""
    lib_path = os.path.join(ROOT, "paper_1304_0681_gb300", "libswgb.so")
    if not os.path.exists(lib_path):
        pytest.skip("libswgb.so not built")
    lib = ctypes.CDLL(lib_path)
    lib.sw_strerror.restype = ctypes.c_char_p
    lib.sw_strerror.argtypes = [ctypes.c_int]
    msg = lib.sw_strerror(_header_codes()["SW_ERR_DEVICE_TIMEOUT"]).decode()
    assert "timed out" in msg
