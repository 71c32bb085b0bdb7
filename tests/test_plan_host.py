"""Host logic of the launch planner (no GPU): the lane-plan cost model that
the planner kernels and plans share (score_plan_of in swgb_internal.h) must
pick, for every read length up to the library's maximum, exactly the plan of
a brute-force search over every (lanes, rows) candidate, and it must honour
overrides.  The program is compiled with the host compiler against the
library's own header."""
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
// brute force: every T = 1..32 for every row count, cost chunks x T x
// (6.5 R + 40) / (G T / 32) in exact integers, the first minimum wins
static void brute(int mode, int m, long hmax, int &lanes, int &ri_best)
{
    const int max_rows = (mode == MODE_I16 && hmax > 510) ? 32 : 64;
    long bn = -1, bd = 1;
    lanes = 32; ri_best = 4;
    for (int ri = 0; ri < N_SCORE_ROWS; ++ri) {
        const int R = score_rows_at(ri);
        if (R > max_rows) continue;
        for (int T = 1; T <= 32; ++T) {
            const int chunks = (m + T * R - 1) / (T * R);
            if (chunks > 1 && T < 32) continue;
            const long G = 32 / T, num = (long)chunks * (13 * R + 80) * 16;
            if (bn < 0 || num * bd < bn * G) { bn = num; bd = G; lanes = T; ri_best = ri; }
        }
    }
}
int main()
{
    int bad = 0;
    for (int mode = 0; mode < N_MODES; ++mode)
        for (int m = 1; m <= SW_MAX_READ_LEN; ++m)
            for (long hmax : {5L * m, 500L}) {
                int l1, r1, l2, r2;
                score_plan_of(mode, m, hmax, nullptr, 0, l1, r1);
                brute(mode, m, hmax, l2, r2);
                if (l1 != l2 || r1 != r2) { if (bad++ < 5) printf("m=%d mode=%d: %d/%d vs %d/%d\n", m, mode, l1, r1, l2, r2); }
            }
    // an override covers classes up to its read length
    PlanOverride ov[2] = {{100, 3, 50}, {300, 32, 8}};
    int l, r;
    score_plan_of(MODE_I16, 90, 450, ov, 2, l, r);
    if (l != 3 || score_rows_at(r) != 50) { printf("override 1: %d %d\n", l, r); ++bad; }
    score_plan_of(MODE_I16W, 250, 1250, ov, 2, l, r);
    if (l != 32 || score_rows_at(r) != 8) { printf("override 2: %d %d\n", l, r); ++bad; }
    // a 50-row plan needs 6-bit row tags: a class whose scores may pass 510 skips it
    PlanOverride ov3[1] = {{100, 2, 50}};
    score_plan_of(MODE_I16, 100, 1000, ov3, 1, l, r);
    if (l == 2 && score_rows_at(r) == 50) { printf("override 3 taken\n"); ++bad; }
    printf("mismatches %d\n", bad);
    return bad != 0;
}
'''


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and CUDA headers")
def test_cost_model_matches_brute_force(tmp_path):
    src = tmp_path / "plan_check.cpp"
    src.write_text(SRC)
    exe = tmp_path / "plan_check"
    inc = os.path.join(ROOT, "paper_1304_0681_gb300", "csrc")
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mismatches 0" in out.stdout
