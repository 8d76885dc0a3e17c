"""The profile test used to compare independent shower samples: it accepts
two oracle samples of the same physics drawn with different seeds, and it
rejects a sample with a planted mistake (lead 5% too dense) -- the mistake is
planted in the oracle's input, on the CPU."""
import numpy as np

from paper_2203_09467_gb300 import workloads as W
from stats_util import profile_test


def sample(oracle_mod, seed, rho_scale=1.0, n=1500):
    s = W.calo_setup(seed=seed)
    s.materials = s.materials.copy()
    s.materials[0, 2] *= rho_scale
    o = oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
    prim = W.calo_primaries(n, energy=2000.0, seed=seed)
    h, sm = o.run(prim, n, np.arange(n))
    return h


def test_profile_test_accepts_same_physics_and_rejects_planted_mistake(oracle_mod):
    a = sample(oracle_mod, 101)
    b = sample(oracle_mod, 202)
    t2, dof, p = profile_test(a, b)
    assert p > 1e-3, (t2, p)
    c = sample(oracle_mod, 303, rho_scale=1.05)
    t2, dof, p = profile_test(a, c)
    assert p < 1e-6, (t2, p)
