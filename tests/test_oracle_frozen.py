"""The oracle's arithmetic is frozen: its per-event results on small samples
of the slab, calorimeter and calorimeter-in-2-T workloads equal the ones
stored in tests/golden/oracle_frozen.txt (written by
tests/golden/make_oracle_frozen.py, which calls only the oracle).  Kernel
changes must agree with the oracle as it stands; a deliberate change of the
oracle's arithmetic rewrites the file in a commit that names the passage,
or the reading of it, that justifies it.  Energies are compared to 1e-12
relative (the C library's transcendental functions may differ in the last
bit between machines), step and track counts exactly."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "oracle_frozen.txt")


def _maker():
    spec = importlib.util.spec_from_file_location("make_oracle_frozen",
                                                  os.path.join(HERE, "golden", "make_oracle_frozen.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_oracle_results_are_the_frozen_ones(oracle_mod):
    stored = {}
    for line in open(GOLD):
        if line.startswith("#"):
            continue
        f = line.split()
        stored.setdefault(f[0], []).append([float.fromhex(v) for v in f[2:6]] + [int(f[6]), int(f[7])])
    m = _maker()
    assert sorted(stored) == sorted(nm for nm, _, _, _ in m.SAMPLES)
    for name, rows in stored.items():
        want = np.array(rows)
        got = m.results(name)
        assert got.shape[0] == want.shape[0], name
        scale = want[:, 3][:, None]  # e_in
        assert np.all(np.abs(got[:, :4] - want[:, :4]) <= 1e-12 * scale), name
        assert np.array_equal(got[:, 4:6].astype(np.int64), want[:, 4:6].astype(np.int64)), name
