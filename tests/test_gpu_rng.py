"""The oracle's Philox4x32-10 against cuRAND's implementation, run on the
GPU (NVIDIA's library as an independent definition of the generator)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcurand_philox.so")
    src = os.path.join(HERE, "csrc", "curand_philox.cu")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, src])
    L = ctypes.CDLL(so)
    L.curand_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    return L


def test_oracle_philox_equals_curand(curand_lib, oracle_mod):
    rng = np.random.default_rng(5)
    n = 2000
    keys = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctrs = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    # the harness reaches counter words (c0, c1) by skipping 4 (c1 2^32 + c0)
    # outputs, which must fit in 64 bits: c1 < 2^30
    ctrs[:, 1] >>= 2
    ctrs[:10] = 0
    keys[:10] = 0
    ctrs[5:10, 0] = np.arange(5)
    out = np.zeros((n, 4), np.uint32)
    assert curand_lib.curand_philox(keys.ctypes.data, ctrs.ctypes.data, n, out.ctypes.data) == 0
    for i in range(n):
        assert np.array_equal(out[i], oracle_mod.philox4x32_10(ctrs[i], keys[i])), i
