"""The step kernels' FP64 division and square root on the integer pipe
(paper_2203_09467_gb300/csrc/emt_intdiv.cuh) compiled as host code and
compared bit for bit with the C division operator and sqrt (IEEE-754, round
to nearest even) on random operands: uniform bit patterns, divisors near
powers of two, equal significands, dividends near 2, nearby exponents and
exact quotients; square roots of any positive double, of significands near
1 and 2 and of exact squares; with the FP32 reciprocal (square root) seed
moved by up to three units of its last place.  The GPU build is compared with the native FP64 division in
tests/test_gpu_intdiv.py."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("intdiv") / "intdiv_host")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "csrc", "intdiv_host.cpp")])
    return exe


def test_integer_division_and_sqrt_equal_ieee(driver):
    n = 4_000_000
    procs = [subprocess.Popen([driver, str(n), str(seed)], stdout=subprocess.PIPE, text=True)
             for seed in range(1, 5)]
    fast = 0
    for p in procs:
        out, _ = p.communicate()
        tot, nf, bad = (int(v) for v in out.split()[-3:])
        assert tot == n
        assert bad == 0, out
        fast += nf
    # most operands take the integer path (the rest are the native division)
    assert fast > 0.85 * 4 * n
