"""The FP64 census build of the oracle (oracle/census.cpp) computes exactly
what the oracle computes, and counts what the step is known to do: one
logarithm per step in matter (the free path), none in vacuum."""
import numpy as np

from paper_2203_09467_gb300 import workloads as W


def test_census_build_equals_oracle(oracle_mod):
    from oracle import census
    s = W.calo_setup()
    n = 6
    prim = W.calo_primaries(n, energy=500.0)
    out, hist, summ = census.census(s, prim, n)
    ref = oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
    rh, rs = ref.run(prim, n, np.arange(n), n_threads=1)
    assert np.array_equal(rs, summ) and np.array_equal(rh, hist)
    per = out["per_track_step"]
    assert out["track_steps"] == rs[:, 4].sum()
    # every step in matter draws its free path with one logarithm; the
    # primaries' first steps start in vacuum
    assert 0.9 < per["log"] <= 1.2
    assert out["flops_per_track_step"] > 10


def test_census_counts_vacuum_steps_without_logarithm(oracle_mod):
    """Photons in a world of vacuum: no cross section, no free path, no log."""
    from oracle import census
    s = W.slab_setup()
    s.materials = np.array([W.VACUUM], np.float64)
    n = 3
    prim = {"event": np.arange(n, dtype=np.int32), "type": np.zeros(n, np.int32), "T": np.full(n, 50.0),
            "pos": np.tile([0.0, 0.0, -1.0], (n, 1)), "dir": np.tile([0.0, 0.0, 1.0], (n, 1))}
    out, hist, summ = census.census(s, prim, n)
    assert out["per_track_step"]["log"] == 0.0
    assert summ[:, 1].sum() == 150.0  # all escaped
