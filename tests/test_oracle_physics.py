"""Pins of the oracle's closed forms against limits, identities, published
constants and numerical quadrature (the paper names the models, Table 1, but
prints no formula; the forms are textbook ones cited in oracle/emt_oracle.c)."""
import os

import numpy as np
import pytest
from scipy import integrate

ME = 0.51099895
RE = 2.8179403262e-13
ALPHA = 1 / 137.035999084
NA = 6.02214076e23
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def L(oracle_mod):
    return oracle_mod.lib()


def quad(f, a, b, **kw):
    v, err = integrate.quad(f, a, b, epsabs=0, epsrel=1e-12, limit=400, **kw)
    return v


def test_radiation_length_matches_pdg(L):
    for line in open(os.path.join(GOLD, "pdg_radiation_length.txt")):
        if line.startswith("#") or not line.strip():
            continue
        Z, A, x0 = map(float, line.split())
        assert abs(L.orc_x0_gcm2(Z, A) / x0 - 1) < 5e-3


def test_klein_nishina_limits(L):
    thomson = 8 * np.pi / 3 * RE ** 2
    # Thomson-limit series sigma_T (1 - 2k + 26/5 k^2 - 133/10 k^3 + 1144/35 k^4)
    # at kappa = 1e-2 (the closed form loses digits to cancellation much
    # below that; photons are transported only above 1 MeV, kappa ~ 2)
    kap = 1e-2
    series = 1 - 2 * kap + 26 / 5 * kap ** 2 - 133 / 10 * kap ** 3 + 1144 / 35 * kap ** 4
    assert abs(L.orc_sigma_kn(kap * ME) / (thomson * series) - 1) < 1e-7
    kap = 1e6
    hi = np.pi * RE ** 2 / kap * (np.log(2 * kap) + 0.5)
    assert abs(L.orc_sigma_kn(kap * ME) / hi - 1) < 1e-4


@pytest.mark.parametrize("k", [0.1, 1.0, 10.0, 1e3, 1e5])
def test_klein_nishina_total_is_integral_of_differential(L, k):
    eps0 = 1 / (1 + 2 * k / ME)
    tot = quad(lambda e: L.orc_dsigma_kn_deps(k, e), eps0, 1.0)
    assert abs(tot / L.orc_sigma_kn(k) - 1) < 1e-9


def test_pair_limits(L):
    for Z, A in [(82, 207.2), (18, 39.948)]:
        unit = A / (L.orc_x0_gcm2(Z, A) * NA)
        assert abs(L.orc_sigma_pair_atom(Z, A, 1e9) / unit - 7 / 9) < 1e-8
        assert L.orc_sigma_pair_atom(Z, A, 2 * ME) == 0.0
        assert L.orc_sigma_pair_atom(Z, A, 1.0) < 0.05 * unit


@pytest.mark.parametrize("k", [1.5, 10.0, 1e3])
def test_pair_total_is_integral_of_differential(L, k):
    e0 = ME / k
    tot = quad(lambda x: L.orc_dsigma_pair_dx(82, 207.2, k, x), e0, 1 - e0)
    assert abs(tot / L.orc_sigma_pair_atom(82, 207.2, k) - 1) < 1e-9


def test_photo_scaling(L):
    s = L.orc_sigma_photo_atom(82, 2.0, 0.088)
    assert abs(L.orc_sigma_photo_atom(82, 4.0, 0.088) / s - 0.5) < 1e-14
    assert abs(L.orc_sigma_photo_atom(41, 2.0, 0.0) / s - 1 / 32) < 1e-14
    assert L.orc_sigma_photo_atom(82, 0.08, 0.088) == 0.0
    # Sauter high-energy K-shell limit x 5/4 written out
    want = 1.25 * 4 * np.pi * RE ** 2 * ALPHA ** 4 * 82 ** 5 * ME / 2.0
    assert abs(s / want - 1) < 1e-13


def test_photo_against_published_lead_attenuation(L):
    """Published value: NIST's total attenuation of lead at 1 MeV (below the
    pair threshold: Compton + photoelectric + a few percent of coherent
    scattering).  The photoelectric model is about 28% of it there, so the
    oracle's Compton + photoelectric sum within 5% of the published total
    pins the photoelectric magnitude to about 18%: a wrong power of alpha
    or Z, a lost 4 pi or the missing 5/4 of the outer shells (-7% of the
    total) all fail.  Measured: -1.7% (the coherent part is not included)."""
    rows = np.loadtxt(os.path.join(GOLD, "nist_lead_attenuation.txt"))
    k, mu_rho = np.atleast_2d(rows)[0]
    Z, A = 82.0, 207.2
    atoms_per_g = 6.02214076e23 / A
    model = (L.orc_sigma_photo_atom(Z, k, 0.088) + Z * L.orc_sigma_kn(k)) * atoms_per_g
    assert abs(model / mu_rho - 1) < 0.05, model / mu_rho
    photo_share = L.orc_sigma_photo_atom(Z, k, 0.088) * atoms_per_g / mu_rho
    assert 0.2 < photo_share < 0.35


def test_brems_energy_integral_is_E_over_X0(L):
    """Complete-screening spectrum: int_0^E k dSigma/dk dk = E / X0."""
    x0 = 0.56
    for T in [10.0, 1e3, 1e5]:
        E = T + ME
        v = quad(lambda k: k * L.orc_dsigma_brems_macro_dk(x0, T, k), 0.0, E)
        assert abs(v / (E / x0) - 1) < 1e-10


@pytest.mark.parametrize("T", [1.5, 20.0, 1e4])
def test_brems_discrete_and_restricted_loss(L, T):
    x0, kc = 0.56, 1.0
    s = quad(lambda k: L.orc_dsigma_brems_macro_dk(x0, T, k), kc, T)
    assert abs(s / L.orc_sigma_brems_macro(x0, T, kc) - 1) < 1e-10
    kp = min(kc, T)
    r = quad(lambda k: k * L.orc_dsigma_brems_macro_dk(x0, T, k), 0.0, kp)
    assert abs(r / L.orc_dedx_rad(x0, T, kc) - 1) < 1e-10
    assert L.orc_sigma_brems_macro(x0, 0.9, kc) == 0.0


def test_moller_symmetry_and_total(L):
    T = 50.0
    for e in [0.01, 0.1, 0.3, 0.45]:
        a, b = L.orc_dsigma_moller_deps(T, e), L.orc_dsigma_moller_deps(T, 1 - e)
        assert abs(a / b - 1) < 1e-13
    for T, cut in [(3.0, 1.0), (100.0, 1.0), (1e4, 1.0)]:
        tot = quad(lambda e: L.orc_dsigma_moller_deps(T, e), cut / T, 0.5)
        assert abs(tot / L.orc_sigma_moller(T, cut) - 1) < 1e-10
    assert L.orc_sigma_moller(2.0, 1.0) == 0.0


def test_bhabha_ultrarelativistic_limit_and_total(L):
    T = 1e8
    norm = 2 * np.pi * RE ** 2 * ME / T
    for e in [0.05, 0.3, 0.7, 0.95]:
        want = (1 - e + e * e) ** 2 / e ** 2
        assert abs(L.orc_dsigma_bhabha_deps(T, e) / norm / want - 1) < 1e-7
    for T, cut in [(1.5, 1.0), (100.0, 1.0), (1e4, 1.0)]:
        tot = quad(lambda e: L.orc_dsigma_bhabha_deps(T, e), cut / T, 1.0)
        assert abs(tot / L.orc_sigma_bhabha(T, cut) - 1) < 1e-10


def test_heitler_dirac_limit_and_total(L):
    T = 1e-7 * ME
    g = 1 + T / ME
    beta = np.sqrt(1 - 1 / g ** 2)
    assert abs(L.orc_sigma_heitler(T) / (np.pi * RE ** 2 / beta) - 1) < 1e-3
    for T in [0.01, 1.0, 100.0, 1e4]:
        tau = T / ME
        emin = 0.5 * (1 - np.sqrt(tau / (tau + 2)))
        tot = quad(lambda e: L.orc_dsigma_heitler_deps(T, e), emin, 1 - emin, points=[emin * 2])
        assert abs(tot / L.orc_sigma_heitler(T) - 1) < 1e-9


@pytest.mark.parametrize("charge", [-1, 1])
@pytest.mark.parametrize("T", [3.0, 30.0, 3e3])
def test_restricted_plus_hard_equals_unrestricted(L, charge, T):
    """S(cut) + n_el int_cut^max T_d dsigma/dT_d dT_d = S(no cut): the
    Berger-Seltzer F(tau, Delta) terms agree with Moller/Bhabha."""
    Z, A, rho, I = 82, 207.2, 11.35, 823.0
    nel = rho * NA / A * Z
    cut = 1.0
    tmax = T / 2 if charge < 0 else T
    f = L.orc_dsigma_moller_deps if charge < 0 else L.orc_dsigma_bhabha_deps
    hard = nel * quad(lambda e: e * T * f(T, e), cut / T, tmax / T)
    s_cut = L.orc_dedx_coll(Z, A, rho, I, charge, T, cut)
    s_all = L.orc_dedx_coll(Z, A, rho, I, charge, T, 2 * T)
    assert abs((s_cut + hard) / s_all - 1) < 1e-9


def test_unrestricted_collision_loss_is_plausible(L):
    """Minimum of the unrestricted electron collision loss in Pb near
    1 MeV cm^2/g (loose sanity; absolute accuracy is parity unpinned)."""
    T = np.logspace(-1, 3, 60)
    s = np.array([L.orc_dedx_coll(82, 207.2, 11.35, 823.0, -1, t, 2 * t) for t in T]) / 11.35
    assert 0.8 < s.min() < 1.3


@pytest.mark.parametrize("Z,A,rho,I", [(82, 207.2, 11.35, 823.0), (18, 39.948, 1.396, 188.0)])
@pytest.mark.parametrize("charge", [-1, 1])
def test_restricted_loss_reaches_the_fermi_plateau(L, Z, A, rho, I, charge):
    """With the high-energy density-effect asymptote, delta = 2 ln(beta
    gamma) + 2 ln(hbar omega_p / I) - 1, the restricted collision loss tends
    to the Fermi plateau 2 pi r_e^2 m n_el ln(2 cut m / (hbar omega_p)^2) as
    T grows with the cut fixed (the tau-dependence of the logarithm, of
    F+-(tau, Delta) and of delta cancel; the constant terms cancel for both
    charges), with hbar omega_p = 28.816 sqrt(rho Z / A) eV."""
    cut = 1.0
    nel = rho * NA / A * Z
    hwp = 28.816e-6 * np.sqrt(rho * Z / A)
    plateau = 2 * np.pi * RE**2 * ME * nel * np.log(2 * cut * ME / hwp**2)
    s = [L.orc_dedx_coll(Z, A, rho, I, charge, T, cut) for T in (1e3, 1e4, 1e5, 1e6)]
    dev = np.abs(np.array(s) / plateau - 1)
    assert dev[-1] < 1e-6
    assert np.all(np.diff(dev) <= 0)  # approaches the plateau monotonically


def test_gauss_legendre(oracle_mod):
    x, w = oracle_mod.gauss_legendre(16)
    xr, wr = np.polynomial.legendre.leggauss(16)
    assert np.max(np.abs(x - xr)) < 1e-14 and np.max(np.abs(w - wr)) < 1e-14
    for p in range(0, 32, 3):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs((w * x ** p).sum() - exact) < 1e-14


@pytest.fixture(scope="module")
def calo(oracle_mod):
    from paper_2203_09467_gb300 import workloads as W
    s = W.calo_setup()
    return oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed), s


def test_tables_match_closed_forms(calo, L):
    o, s = calo
    grid = o.grid()
    assert len(grid) == 65
    assert abs(grid[0] - 1e-3) < 1e-18 and abs(grid[-1] / 1e5 - 1) < 1e-15
    assert abs(grid[24] - 1.0) < 1e-15
    Z, A, rho, I, bk = s.materials[0]
    nat = rho * NA / A
    x0 = L.orc_x0_gcm2(Z, A) / rho
    i = 40
    E = grid[i]
    assert abs(o.table(0, 0, 1)[i] / (Z * nat * L.orc_sigma_kn(E)) - 1) < 1e-14
    assert abs(o.table(0, 0, 2)[i] / (nat * L.orc_sigma_pair_atom(Z, A, E)) - 1) < 1e-13
    assert abs(o.table(0, 1, 1)[i] / L.orc_sigma_brems_macro(x0, E, 1.0) - 1) < 1e-14
    assert abs(o.table(0, 2, 2)[i] / (Z * nat * L.orc_sigma_heitler(E)) - 1) < 1e-14


@pytest.mark.parametrize("m,p", [(0, 1), (0, 2), (1, 1), (1, 2)])
def test_range_table_is_integral_of_inverse_dedx(calo, L, m, p):
    o, s = calo
    Z, A, rho, I, bk = s.materials[m]
    x0 = L.orc_x0_gcm2(Z, A) / rho
    charge = -1 if p == 1 else 1

    def S(E):
        return L.orc_dedx_coll(Z, A, rho, I, charge, E, 1.0) + L.orc_dedx_rad(x0, E, 1.0)

    grid = o.grid()
    R = o.table(m, p, 3)
    assert abs(R[0] / (grid[0] / S(grid[0])) - 1) < 1e-14
    for n in [8, 24, 40, 64]:
        # adaptive quadrature of 1/S(E) in E, interval by interval
        want = grid[0] / S(grid[0]) + sum(quad(lambda E: 1.0 / S(E), grid[i - 1], grid[i])
                                          for i in range(1, n + 1))
        assert abs(R[n] / want - 1) < 1e-10
    # exact inverse of the piecewise-linear range
    for T in [1.0, 3.7, 250.0, 9999.0]:
        r = o.range(m, p, T)
        assert abs(o.inv_range(m, p, r) / T - 1) < 1e-12
