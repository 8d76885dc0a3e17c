"""Pins of the oracle's Rayleigh scattering (screened-atom form factor) and
Sauter photoelectron angle.

The atomic Rayleigh cross section must equal the numerical integral of its
differential form over both branches of its evaluation (Taylor series and
closed form), reduce to Z^2 times the Thomson cross section at low energy
(coherent scattering off Z free charges) and fall as 1/k^2 at high energy
(the form factor cuts the angles off at q a ~ 1); the angle samplers must
follow their densities (KS tests against numerically integrated
cumulative distributions); a photon whose only process is Rayleigh keeps
its energy and changes direction."""
import numpy as np
import pytest
from scipy import integrate, stats

from paper_2203_09467_gb300 import workloads as W

ME = 0.51099895
RE = 2.8179403262e-13


@pytest.mark.parametrize("Z", [6.0, 14.0, 82.0])
def test_rayleigh_total_is_integral_of_differential(oracle_mod, Z):
    L = oracle_mod.lib()
    for k in np.logspace(-3.3, 2, 23):  # b from ~1e-3 (series) to ~1e8 (closed form)
        f = lambda x: L.orc_dsigma_rayleigh_dx(Z, k, x)
        pts = [min(2.0, 10.0 ** e) for e in range(-9, 1)]
        num = integrate.quad(f, 0.0, 2.0, points=pts, epsabs=0, epsrel=1e-12, limit=400)[0]
        assert abs(L.orc_sigma_rayleigh_atom(Z, k) / num - 1) < 1e-9, (Z, k)


def test_rayleigh_limits(oracle_mod):
    L = oracle_mod.lib()
    thomson = 8 * np.pi / 3 * RE ** 2
    for Z in (6.0, 82.0):
        assert abs(L.orc_sigma_rayleigh_atom(Z, 1e-7) / (Z * Z * thomson) - 1) < 1e-6
        r = L.orc_sigma_rayleigh_atom(Z, 1e4) / L.orc_sigma_rayleigh_atom(Z, 1e3)
        assert abs(r / 0.01 - 1) < 1e-3


def cdf_from(pdf, lo, hi, points=None):
    tot = integrate.quad(pdf, lo, hi, points=points, epsabs=0, epsrel=1e-11, limit=400)[0]

    def cdf(x):
        pts = None if points is None else [p for p in points if lo < p < x]
        return integrate.quad(pdf, lo, x, points=pts or None, epsabs=0, epsrel=1e-10, limit=400)[0] / tot
    return cdf


@pytest.mark.parametrize("k", [0.02, 0.3, 3.0])
def test_rayleigh_angle_follows_density(oracle_mod, k):
    L = oracle_mod.lib()
    Z = 82.0
    cdf = cdf_from(lambda x: L.orc_dsigma_rayleigh_dx(Z, k, x), 0.0, 2.0,
                   points=[10.0 ** e for e in range(-9, 0)])
    n = 3000
    u = np.empty(n)
    for i in range(n):
        out = oracle_mod.sample(oracle_mod.RAYLEIGH, k, Z, 1.0, 4, 5, i + 1)
        assert out[0] == k and out[4] == 0  # energy kept, no secondary
        u[i] = cdf(min(2.0, 1.0 - out[3]))
    assert stats.kstest(u, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("T", [0.5, 2.0, 20.0])
def test_sauter_angle_follows_density(oracle_mod, T):
    E = T + ME
    b = np.sqrt(T * (T + 2 * ME)) / E
    g = E / ME
    pdf = lambda c: (1 - c * c) / (1 - b * c) ** 4 * (1 + 0.5 * g * (g - 1) * (g - 2) * (1 - b * c))
    cdf = cdf_from(pdf, -1.0, 1.0)
    bk = 0.088
    n = 2500
    u = np.empty(n)
    for i in range(n):
        out = oracle_mod.sample(oracle_mod.PHOTO_ANGULAR, T + bk, bk, 1.0, 6, 7, i + 1)
        assert abs(out[6] - T) < 1e-12
        u[i] = cdf(out[9])
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_rayleigh_only_photon_keeps_energy(oracle_mod):
    s = W.slab_setup(mask=oracle_mod.RAYLEIGH_BIT, thickness=1e4)
    s.world[3:9] = [-1e5, -1e5, -1e5, 1e5, 1e5, 1e5]
    s.world[1] = s.world[2] = 1e4
    o = oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
    turned = 0
    for i in range(300):
        t = np.array([0, 0.05, 0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0, 0], float)
        t2, sec, info = o.step_one(t, i + 1, 3)
        assert info[3] == 1 and info[4] == 9 and len(sec) == 0
        assert t2[1] == 0.05 and abs(np.linalg.norm(t2[5:8]) - 1) < 1e-14
        turned += t2[7] < 0.999
    assert turned > 100
