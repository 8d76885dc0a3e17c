"""The premise of the step kernels' integer-pipe comparisons: for IEEE
doubles and floats that are not NaN, the signed order of the bit patterns is
the numeric order whenever at least one operand is > 0; `x > 0` is the
pattern being > 0 and `x != 0` is the pattern without its sign bit being
nonzero, for every value.  Checked here on the host over random values of
every class (zeros of both signs, subnormals, normals, infinities), so a
call site that meets the condition is exact."""
import numpy as np


def _values(dtype, n, rng):
    info = np.finfo(dtype)
    mags = np.concatenate([
        np.zeros(8),
        rng.uniform(0, 1, n) * info.smallest_subnormal * 64,   # subnormals
        10.0 ** rng.uniform(np.log10(info.tiny), np.log10(info.max) - 1, n),
        rng.uniform(0, 10, n),
        np.array([info.tiny, info.max, np.inf, info.smallest_subnormal, 1.0]),
    ]).astype(dtype)
    signs = rng.choice(np.array([-1, 1], dtype=dtype), size=mags.size)
    v = (mags * signs).astype(dtype)
    v[:4] = dtype(0.0)
    v[4:8] = -dtype(0.0)
    return v


def _check(dtype, itype):
    rng = np.random.default_rng(7)
    a = _values(dtype, 3000, rng)
    b = _values(dtype, 3000, rng)
    rng.shuffle(b)
    n = min(a.size, b.size)
    a, b = a[:n], b[:n]
    # all pairs of a sample, plus the paired arrays
    s = np.concatenate([a[:400], b[:400]])
    A = np.repeat(s, s.size)
    B = np.tile(s, s.size)
    A = np.concatenate([A, a])
    B = np.concatenate([B, b])
    ia, ib = A.view(itype), B.view(itype)
    ok = (A > 0) | (B > 0)
    assert ok.sum() > 100_000
    assert np.array_equal((ia < ib)[ok], (A < B)[ok])
    assert np.array_equal((ia <= ib)[ok], (A <= B)[ok])
    # the condition matters: two negatives order the other way round
    neg = (A < 0) & (B < 0) & (A != B)
    assert np.any((ia < ib)[neg] != (A < B)[neg])
    # sign and zero tests, every value
    assert np.array_equal(A.view(itype) > 0, A > 0)
    bits = A.view(itype.replace("i", "u"))
    assert np.array_equal((bits << np.array(1, bits.dtype)) != 0, A != 0)


def test_double_bit_order():
    _check(np.float64, "i8")


def test_float_bit_order():
    _check(np.float32, "i4")
