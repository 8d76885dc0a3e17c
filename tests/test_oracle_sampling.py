"""Brute-force histogram pins of the oracle's interaction samplers: each
sampled distribution is compared by chi-square with the binned integral of
the differential cross section it should follow, and every sample is checked
for energy and momentum conservation."""
import numpy as np
import pytest
from scipy import integrate, stats

ME = 0.51099895
SEED, EVENT = 11, 77


def draw_many(oracle_mod, process, E, n, cut_e=1.0, cut_g=1.0):
    return np.array([oracle_mod.sample(process, E, cut_e, cut_g, SEED, EVENT, uid + 1)
                     for uid in range(n)])


def chi2_p(samples, edges, pdf):
    counts, _ = np.histogram(samples, bins=edges)
    w = np.array([integrate.quad(pdf, a, b, epsrel=1e-10)[0] for a, b in zip(edges[:-1], edges[1:])])
    expected = w / w.sum() * len(samples)
    keep = expected > 5
    chi2 = ((counts[keep] - expected[keep]) ** 2 / expected[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


N = 60000


@pytest.mark.parametrize("k", [1.5, 20.0, 2000.0])
def test_compton_spectrum_and_kinematics(oracle_mod, k):
    L = oracle_mod.lib()
    out = draw_many(oracle_mod, oracle_mod.COMPTON, k, N)
    eps = out[:, 0] / k
    kap = k / ME
    e0 = 1 / (1 + 2 * kap)
    assert eps.min() >= e0 * (1 - 1e-12) and eps.max() <= 1.0
    edges = e0 * (1 / e0) ** np.linspace(0, 1, 41)
    assert chi2_p(eps, edges, lambda e: L.orc_dsigma_kn_deps(k, e)) > 1e-3
    # photon angle from two-body kinematics; electron balances momentum
    cost = out[:, 3]
    assert np.allclose(cost, 1 - (1 - eps) / (kap * eps), rtol=0, atol=1e-12)
    sub = out[:2000]
    for o in sub:
        if o[4] == 0:
            continue
        Te = o[6]
        assert abs((o[0] + Te) / k - 1) < 1e-14
        pe = np.sqrt(Te * (Te + 2 * ME))
        p = o[0] * o[1:4] + pe * o[7:10]
        assert np.allclose(p, [0, 0, k], rtol=0, atol=1e-9 * k)


@pytest.mark.parametrize("k", [1.5, 10.0, 5000.0])
def test_pair_spectrum_and_energy(oracle_mod, k):
    L = oracle_mod.lib()
    out = draw_many(oracle_mod, oracle_mod.PAIR, k, N)
    assert np.all(out[:, 4] == 2) and np.all(out[:, 5] == 1) and np.all(out[:, 10] == 2)
    x = (out[:, 6] + ME) / k
    e0 = ME / k
    edges = np.linspace(e0, 1 - e0, 31)
    assert chi2_p(x, edges, lambda v: L.orc_dsigma_pair_dx(82, 207.2, k, v)) > 1e-3
    tot = out[:, 6] + out[:, 11] + 2 * ME
    assert np.max(np.abs(tot / k - 1)) < 1e-14


@pytest.mark.parametrize("T", [3.0, 100.0, 1e4])
def test_brems_spectrum(oracle_mod, T):
    L = oracle_mod.lib()
    kc = 1.0
    out = draw_many(oracle_mod, oracle_mod.BREMS, T, N, cut_g=kc)
    kk = out[:, 6]
    assert kk.min() >= kc and kk.max() <= T * (1 + 1e-14)
    assert np.max(np.abs((out[:, 0] + kk) / T - 1)) < 1e-14
    edges = kc * (T / kc) ** np.linspace(0, 1, 31)
    assert chi2_p(kk, edges, lambda k: L.orc_dsigma_brems_macro_dk(0.56, T, k)) > 1e-3


@pytest.mark.parametrize("T", [2.5, 50.0, 1e4])
def test_moller_spectrum_and_momentum(oracle_mod, T):
    L = oracle_mod.lib()
    cut = 1.0
    out = draw_many(oracle_mod, oracle_mod.IONI, T, N, cut_e=cut)
    eps = out[:, 6] / T
    assert eps.min() >= cut / T * (1 - 1e-14) and eps.max() <= 0.5 + 1e-14
    edges = (cut / T) * (0.5 * T / cut) ** np.linspace(0, 1, 31)
    assert chi2_p(eps, edges, lambda e: L.orc_dsigma_moller_deps(T, e)) > 1e-3
    for o in out[:2000]:
        Tn, Td = o[0], o[6]
        assert abs((Tn + Td) / T - 1) < 1e-14
        p = np.sqrt(Tn * (Tn + 2 * ME)) * o[1:4] + np.sqrt(Td * (Td + 2 * ME)) * o[7:10]
        # the parent direction is set by momentum balance with |p| fixed
        # by the kinematics; the balance holds to the direction rounding
        assert np.allclose(p, [0, 0, np.sqrt(T * (T + 2 * ME))], rtol=0, atol=1e-9 * T)


@pytest.mark.parametrize("T", [1.5, 50.0, 1e4])
def test_bhabha_spectrum(oracle_mod, T):
    L = oracle_mod.lib()
    cut = 1.0
    out = draw_many(oracle_mod, oracle_mod.BHABHA, T, N, cut_e=cut)
    eps = out[:, 6] / T
    assert eps.min() >= cut / T * (1 - 1e-14) and eps.max() <= 1.0 + 1e-14
    edges = (cut / T) * (T / cut) ** np.linspace(0, 1, 31)
    assert chi2_p(eps, edges, lambda e: L.orc_dsigma_bhabha_deps(T, e)) > 1e-3


def test_bhabha_rejection_function_bounded(oracle_mod):
    """The acceptance function beta^2 eps^2 (bracket) stays in [0, 1]."""
    L = oracle_mod.lib()
    RE = 2.8179403262e-13
    for T in [1.01, 2.0, 10.0, 1e3, 1e6]:
        eps = np.linspace(1.0 / T, 1.0, 2001)
        tau = T / ME
        b2 = tau * (tau + 2) / (tau + 1) ** 2
        f = np.array([L.orc_dsigma_bhabha_deps(T, e) for e in eps]) * T / (2 * np.pi * RE ** 2 * ME) * b2 * eps ** 2
        assert f.max() <= 1 + 1e-12 and f.min() >= 0


@pytest.mark.parametrize("T", [1.0, 30.0, 3000.0])
def test_annihilation_spectrum_and_conservation(oracle_mod, T):
    L = oracle_mod.lib()
    out = draw_many(oracle_mod, oracle_mod.ANNIH, T, N)
    Et = T + 2 * ME
    eps = out[:, 6] / Et
    tau = T / ME
    emin = 0.5 * (1 - np.sqrt(tau / (tau + 2)))
    edges = emin * ((1 - emin) / emin) ** np.linspace(0, 1, 31)
    assert chi2_p(eps, edges, lambda e: L.orc_dsigma_heitler_deps(T, e)) > 1e-3
    assert np.max(np.abs((out[:, 6] + out[:, 11]) / Et - 1)) < 1e-14
    p0 = np.sqrt(T * (T + 2 * ME))
    for o in out[:2000]:
        p = o[6] * o[7:10] + o[11] * o[12:15]
        assert np.allclose(p, [0, 0, p0], rtol=0, atol=1e-9 * Et)
