"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al. SC'11)."""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.replace("->", " ").split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle_mod.philox4x32_10(ctr, key)
        assert list(map(int, got)) == want


def test_uniform_is_open_interval_and_uniform(oracle_mod):
    u = np.array([oracle_mod.track_uniform(7, 3, 11, s, j) for s in range(200) for j in range(50)])
    assert np.all(u > 0.0) and np.all(u < 1.0)
    # moments of U(0,1) for 10,000 draws: mean 1/2 +- 4 sigma, var 1/12
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.005
    # 20-bin chi-square
    h, _ = np.histogram(u, bins=20, range=(0, 1))
    chi2 = ((h - u.size / 20) ** 2 / (u.size / 20)).sum()
    assert chi2 < 45  # chi2(19) 0.999 quantile ~ 43.8


def test_draw_layout_matches_block_words(oracle_mod):
    """Draw j uses block j>>1, words 2(j&1), 2(j&1)+1 of that block."""
    seed, ev, uid, step = 5, (3 << 32) | 17, (9 << 32) | 123, 42
    key = [ev & 0xFFFFFFFF, (ev >> 32) ^ seed]
    for j in range(6):
        out = oracle_mod.philox4x32_10([uid & 0xFFFFFFFF, uid >> 32, step, j >> 1], key)
        lo, hi = int(out[2 * (j & 1)]), int(out[2 * (j & 1) + 1])
        w = (hi << 32) | lo
        want = ((w >> 12) + 0.5) * 2.0 ** -52
        assert oracle_mod.track_uniform(seed, ev, uid, step, j) == want


def test_streams_differ(oracle_mod):
    a = [oracle_mod.track_uniform(1, 0, 1, 0, j) for j in range(8)]
    b = [oracle_mod.track_uniform(1, 0, 2, 0, j) for j in range(8)]
    c = [oracle_mod.track_uniform(1, 0, 1, 1, j) for j in range(8)]
    d = [oracle_mod.track_uniform(1, 1, 1, 0, j) for j in range(8)]
    assert len({tuple(a), tuple(b), tuple(c), tuple(d)}) == 4
    kids = {oracle_mod.child_uid(1, 0, 1, s, k) for s in range(100) for k in range(2)}
    assert len(kids) == 200
