"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host only).

oracle/sanitize_main.c drives every oracle entry point over small and
degenerate clouds (duplicates, exact ties, extreme scales, one and two
points, invalid arguments); built with the oracle source under ASan + UBSan
it must run to completion with no report, and every RadiusFPS switch
combination must reproduce plain FPS.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path, openmp):
    exe = str(tmp_path / ("oracle_san_omp" if openmp else "oracle_san"))
    cmd = ["gcc", "-std=c11", "-g", "-O1", "-ffp-contract=off", "-fno-fast-math",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
           os.path.join(ROOT, "oracle", "rfps_oracle.c"), os.path.join(ROOT, "oracle", "sanitize_main.c"),
           "-o", exe, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    if r.returncode != 0:
        if "sanitize" in r.stderr or "asan" in r.stderr.lower():
            pytest.skip("gcc without sanitizer runtimes: " + r.stderr.strip().splitlines()[-1])
        raise AssertionError(r.stderr)
    return exe


@pytest.mark.parametrize("openmp", [False, True], ids=["serial", "openmp"])
def test_oracle_runs_clean_under_asan_and_ubsan(tmp_path, openmp):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = _build(tmp_path, openmp)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", OMP_NUM_THREADS="4")
    r = subprocess.run([exe], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "all checks held" in r.stdout
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr
