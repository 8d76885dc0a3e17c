"""Pins of the oracle's multiple scattering (Highland width, Gaussian
projected angles) and of the dipole angular distributions of
bremsstrahlung photons and pair leptons.

Highland's formula reduces exactly to theta0 = 13.6 MeV / p when the path
is one radiation length times beta^2 (its logarithm vanishes); the
deflection sampler must give projected angles that are Gaussian with that
width (KS test); the dipole sampler must follow dN/dcos ~ (1 - beta cos)^-2,
whose cumulative distribution is integrated numerically here (KS test on the
probability-integral transform); the angular option must leave every
sampled energy unchanged; in a transport step the deflection uses the
pre-step energy, the step length and the material's X0."""
import numpy as np
import pytest
from scipy import integrate, stats

from paper_2203_09467_gb300 import workloads as W

ME = 0.51099895


def beta_of(T):
    return np.sqrt(T * (T + 2 * ME)) / (T + ME)


@pytest.mark.parametrize("T", [2.0, 30.0, 1000.0, 5e4])
def test_highland_at_one_radiation_length(oracle_mod, T):
    x0 = 0.5612
    b = beta_of(T)
    p = np.sqrt(T * (T + 2 * ME))
    assert abs(oracle_mod.highland(T, x0 * b * b, x0) / (13.6 / p) - 1) < 1e-14


def test_highland_trends(oracle_mod):
    x0 = 14.0
    s = np.logspace(-6, 1.5, 40)
    th = np.array([oracle_mod.highland(100.0, v, x0) for v in s])
    assert np.all(np.diff(th) > 0)
    Ts = np.logspace(0, 4, 30)
    th = np.array([oracle_mod.highland(T, 0.1, x0) for T in Ts])
    assert np.all(np.diff(th) < 0)
    assert oracle_mod.highland(100.0, 1e-14, x0) == 0.0  # bracket negative: no deflection


@pytest.mark.parametrize("T,s", [(1000.0, 0.2), (50.0, 0.01)])
def test_msc_projected_angles_are_gaussian(oracle_mod, T, s):
    x0 = 0.5612
    th0 = oracle_mod.highland(T, s, x0)
    n = 20000
    px = np.empty(n)
    py = np.empty(n)
    for i in range(n):
        d = oracle_mod.msc(T, s, x0, [0.0, 0.0, 1.0], 7, 11, i + 1, 3)
        assert abs(np.linalg.norm(d) - 1) < 1e-14
        px[i] = np.arctan2(d[0], d[2])
        py[i] = np.arctan2(d[1], d[2])
    # small angles: the projections are N(0, theta0^2), independent
    assert stats.kstest(px / th0, "norm").pvalue > 1e-3
    assert stats.kstest(py / th0, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(px, py)[0, 1]) < 0.03


def dipole_cdf(x, b):
    f = lambda t: (1 - b * t) ** -2
    tot = integrate.quad(f, -1, 1, epsabs=0, epsrel=1e-12)[0]
    return integrate.quad(f, -1, x, epsabs=0, epsrel=1e-12, points=[1.0])[0] / tot


def test_brems_photon_angle_follows_dipole(oracle_mod):
    T = 2.0
    b = beta_of(T)
    n = 4000
    u = np.empty(n)
    for i in range(n):
        out = oracle_mod.sample(oracle_mod.BREMS_ANGULAR, T, 1.0, 0.1, 5, 9, i + 1)
        cost = out[9]  # photon direction z (parent along +z)
        u[i] = dipole_cdf(min(cost, 1.0), b)
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_pair_lepton_angles_follow_dipole(oracle_mod):
    k = 6.0
    n = 3000
    u = []
    for i in range(n):
        out = oracle_mod.sample(oracle_mod.PAIR_ANGULAR, k, 1.0, 1.0, 5, 9, i + 1)
        dm, dp = out[7:10], out[12:15]
        # azimuths opposite: transverse parts antiparallel
        cross = dm[0] * dp[1] - dm[1] * dp[0]
        dot = dm[0] * dp[0] + dm[1] * dp[1]
        assert abs(cross) <= 1e-12 * (np.hypot(dm[0], dm[1]) * np.hypot(dp[0], dp[1]) + 1e-300) + 1e-15
        assert dot <= 1e-15
        for T, d in ((out[6], dm), (out[11], dp)):
            if T > 0:
                u.append(dipole_cdf(min(d[2], 1.0), beta_of(T)))
    assert stats.kstest(np.array(u), "uniform").pvalue > 1e-3


@pytest.mark.parametrize("proc,ang,E,cg", [(4, 7, 500.0, 1.0), (2, 8, 300.0, 1.0)])
def test_angular_option_keeps_energies(oracle_mod, proc, ang, E, cg):
    for i in range(200):
        a = oracle_mod.sample(proc, E, 1.0, cg, 3, 4, i + 1)
        b = oracle_mod.sample(ang, E, 1.0, cg, 3, 4, i + 1)
        assert a[0] == b[0] and a[6] == b[6] and a[11] == b[11]


def test_msc_in_a_transport_step(oracle_mod):
    """1 GeV e- crossing a 0.5 mm Pb foil in one step (ionisation and
    multiple scattering only): the exit directions scatter with the Highland
    width of the pre-step energy over the foil thickness."""
    s = W.slab_setup(mask=8 + oracle_mod.MSC, thickness=0.05)  # ionisation + msc
    o = oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
    x0 = oracle_mod.lib().orc_x0_gcm2(82.0, 207.2) / 11.35
    T = 1000.0
    th0 = oracle_mod.highland(T, 0.05, x0)
    px = []
    for i in range(6000):
        t = np.array([1, T, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0, 0], float)
        t2, sec, info = o.step_one(t, i + 1, 5)
        if info[2] != 1 or info[3] != 0:  # keep the steps that cross the foil
            continue
        assert abs(info[0] - 0.05) < 1e-15
        px.append(np.arctan2(t2[5], t2[7]))
    px = np.array(px)
    assert len(px) > 5000
    assert stats.kstest(px / th0, "norm").pvalue > 1e-3
