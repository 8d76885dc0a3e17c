"""The step kernels' FP64 logarithm on the integer pipe
(paper_2203_09467_gb300/csrc/emt_intlog.cuh), compiled as host code:
its reduction table equals the one its generator computes in exact
rational arithmetic; on uniforms in (0, 1), arguments next to 1 on both
sides and arbitrary positive normals it never differs from the C library's
log by more than one unit in the last place; and where the two differ, a
240-bit reference (mpmath) says which one is correctly rounded."""
import importlib.util
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2203_09467_gb300", "csrc")


def test_log_table_is_the_generators_output():
    spec = importlib.util.spec_from_file_location("gen_logtab", os.path.join(CSRC, "gen_logtab.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    inv, t, ln2 = gen.table()
    text = open(os.path.join(CSRC, "emt_logtab.h")).read()

    def block(name):
        body = text.split(f"#define {name} {{")[1].split("}")[0]
        return [int(v.rstrip("ul"), 0) for v in re.findall(r"0x[0-9A-F]+ull|\d+u", body)]

    assert block("EMT_LOGTAB_INV") == inv
    hi, lo = block("EMT_LOGTAB_HI"), block("EMT_LOGTAB_LO")
    for j in range(192):
        v = (hi[j] << 64) | lo[j]
        assert (v - (1 << 128) if v >> 127 else v) == t[j]
    # spot values: ln 2 and ln(2^15 / I) against the float library
    import math
    assert abs(ln2 / 2.0 ** 116 - math.log(2.0)) < 1e-16
    for j in (0, 50, 100, 191):
        assert abs(t[j] / 2.0 ** 116 - math.log(32768.0 / inv[j])) < 4e-16
    # |r| bound of the reduction: X I 2^-15 - 1 over each interval
    for j in range(192):
        lo_x, hi_x = 0.75 + j / 256, 0.75 + (j + 1) / 256
        bound = 2 ** -8 if j in (63, 64) else 2 ** -8.4
        assert max(abs(lo_x * inv[j] / 32768 - 1), abs(hi_x * inv[j] / 32768 - 1)) <= bound


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("intlog") / "intlog_host")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "csrc", "intlog_host.cpp")])
    return exe


def test_integer_log_against_libm_and_a_high_precision_reference(driver, tmp_path):
    n = 2_000_000
    path = str(tmp_path / "diff.txt")
    out = subprocess.run([driver, str(n), "400", path], capture_output=True, text=True, check=True).stdout
    tot, diff, big = (int(v) for v in out.split())
    assert tot == n
    assert big == 0          # never more than one unit in the last place apart
    assert diff < 1e-3 * n   # the two agree almost always
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 240
    rows = [[float.fromhex(v) for v in line.split()] for line in open(path)]
    ours = sum(b == float(mpmath.log(mpmath.mpf(x))) for x, a, b in rows)
    # where they differ, the integer path is the correctly rounded one
    assert ours >= 0.99 * len(rows)
