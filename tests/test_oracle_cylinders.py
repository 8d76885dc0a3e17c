"""Pins of the oracle's cylinder-shell geometry (the paper's Sec. 3.2 test
problem: concentric single-element shells about the z axis), of scoring
along z and of the steps-per-track histogram.

The exit distances are checked against brute force (the exit point lies on
the surface the oracle names, every point of the path before it lies inside
the shell, and the point just beyond it is located in the next volume),
against hand-worked distances, and by counting the surfaces a straight
photon crosses when no process is active."""
import numpy as np
import pytest

from paper_2203_09467_gb300 import workloads as W

R = (0.0,) + W.CMS_RADII
H = W.CMS_HALF_Z


def make(oracle_mod, s):
    return oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)


def rho(p):
    return float(np.hypot(p[0], p[1]))


@pytest.mark.parametrize("p,d,t,nxt", [
    ([0, 0, 0], [1, 0, 0], 30.0, 1),                          # leaves the vacuum core
    ([0, 0, 0], [0, 0, 1], H, -2),                            # end plane
    ([0, 0, 0], [0, 0, -1], H, -2),
    ([100, 0, 0], [-1, 0, 0], 70.0, 0),                       # inward onto r = 30
    ([0, 100, 0], [1, 0, 0], 75.0, 2),                        # sqrt(125^2 - 100^2)
    ([50, 40, 0], [-1, 0, 0], 50.0 + np.sqrt(125.0 ** 2 - 40.0 ** 2), 2),  # misses r = 30
    ([350, 0, 0], [1, 0, 0], 25.0, -2),                       # outermost shell
    ([0, 200, 650], [0, 0.6, 0.8], 62.5, -2),                 # end plane before r = 275
])
def test_exit_hand_worked(oracle_mod, p, d, t, nxt):
    o = make(oracle_mod, W.cms_setup(mask=0))
    vol = o.locate(p)
    tt, n = o.nav_exit(vol, p, d)
    assert n == nxt
    assert abs(tt - t) < 1e-12 * max(1.0, t)


def test_locate(oracle_mod):
    o = make(oracle_mod, W.cms_setup(mask=0))
    assert o.locate([0, 0, 0]) == 0
    assert o.locate([29.999, 0, 0]) == 0
    assert o.locate([30.0, 0, 0]) == 1
    assert o.locate([0, -124.0, 600.0]) == 1
    assert o.locate([200.0 / np.sqrt(2), 200.0 / np.sqrt(2), 0]) == 3
    assert o.locate([374.0, 0, -H]) == 5
    assert o.locate([375.0, 0, 0]) == -2
    assert o.locate([0, 0, H + 1e-9]) == -2


def test_exit_brute_force(oracle_mod):
    """Random points in every shell, random directions (some nearly axial,
    some nearly tangent): the exit point is on the named surface, the path
    before it stays in the shell, the point beyond it is in the next volume."""
    o = make(oracle_mod, W.cms_setup(mask=0))
    rng = np.random.default_rng(11)
    n_checked = 0
    for vol in range(6):
        for _ in range(400):
            r = np.sqrt(rng.uniform(R[vol] ** 2, R[vol + 1] ** 2))
            phi = rng.uniform(0, 2 * np.pi)
            p = np.array([r * np.cos(phi), r * np.sin(phi), rng.uniform(-H, H)])
            kind = rng.integers(0, 3)
            if kind == 0:
                d = rng.normal(size=3)
            elif kind == 1:   # nearly along z
                d = np.array([rng.normal() * 1e-3, rng.normal() * 1e-3, rng.choice([-1.0, 1.0])])
            else:             # nearly tangent to the circle through p
                d = np.array([-np.sin(phi), np.cos(phi), rng.normal() * 0.01]) + rng.normal(size=3) * 1e-4
            d /= np.linalg.norm(d)
            if o.locate(p) != vol:
                continue
            t, nxt = o.nav_exit(vol, p, d)
            assert t > 0
            q = p + t * d
            tol = 1e-9 * max(1.0, t)
            if nxt == vol + 1 or (nxt == -2 and abs(abs(q[2]) - H) > tol):
                assert abs(rho(q) - R[vol + 1]) < tol, (vol, p, d, t)
            elif nxt == vol - 1:
                assert abs(rho(q) - R[vol]) < tol
            else:
                assert nxt == -2 and abs(abs(q[2]) - H) < tol
            for f in np.linspace(0, 1, 41)[1:-1]:
                x = p + f * t * d
                assert R[vol] - tol <= rho(x) <= R[vol + 1] + tol and abs(x[2]) <= H + tol
            beyond = o.locate(q + min(1e-6, 1e-7 * t) * d)
            assert beyond == nxt
            n_checked += 1
    assert n_checked > 2000


def test_straight_photons_count_surfaces(oracle_mod):
    """No process active: an isotropic photon from the origin crosses the
    shells until it leaves through r = 375 cm or an end plane; the step count
    is the number of surfaces it meets, counted here from the polar angle."""
    s = W.cms_setup(mask=0)
    o = make(oracle_mod, s)
    prim = W.cms_primaries(1, 500, energy=50.0, seed=3)
    ev = np.arange(500, dtype=np.int32)
    prim = dict(prim, event=ev)
    hist, summ = o.run(prim, 500, np.arange(500))
    for i in range(500):
        d = prim["dir"][i]
        st = np.hypot(d[0], d[1])
        # path length to each radius and to the end plane
        s_end = H / abs(d[2]) if d[2] != 0 else np.inf
        s_r = [r / st if st > 0 else np.inf for r in W.CMS_RADII]
        steps = 1 + sum(1 for x in s_r[:-1] if x < s_end)
        assert summ[i, 4] == steps
        assert summ[i, 1] == 50.0 and summ[i, 0] == 0.0


def test_z_scoring_bins(oracle_mod):
    """Primaries below the cut deposit at their starting point: the energy
    lands in bin floor((z + H) * n_bins / 2H)."""
    s = W.cms_setup()
    o = make(oracle_mod, s)
    zs = [-H + 1.0, -5.0, 0.0, 5.0, 4.999, 699.9, 123.4]
    n = len(zs)
    prim = {"event": np.arange(n, dtype=np.int32), "type": np.full(n, 1, np.int32),
            "T": np.full(n, 0.5), "pos": np.array([[50.0, 0.0, z] for z in zs]),
            "dir": np.tile([0.0, 0.0, 1.0], (n, 1))}
    hist, summ = o.run(prim, n, np.arange(n))
    scale = s.n_bins / (2 * H)
    for i, z in enumerate(zs):
        b = int(np.floor((z + H) * scale))
        assert hist[i, b] == 0.5 and hist[i].sum() == 0.5


def test_cms_ledger_and_step_histogram(oracle_mod):
    s = W.cms_setup()
    o = make(oracle_mod, s)
    n = 6
    prim = W.cms_primaries(n, 20)
    hist, summ, sh = o.run(prim, n, np.arange(n), step_bins=100000)
    # energy ledger per event; the z range covers the whole world
    assert np.allclose(summ[:, 0] + summ[:, 1] + summ[:, 2], summ[:, 3], rtol=1e-12)
    assert np.allclose(hist.sum(1), summ[:, 0], rtol=1e-12)
    # every transported track is counted once with its number of steps
    assert sh.sum() == summ[:, 5].sum()
    assert (sh * np.arange(sh.shape[1])).sum() == summ[:, 4].sum()
    assert sh[:, 0].sum() == 0  # every track takes at least one step
    # photons from the origin take one step to reach r = 30 cm at least
    assert sh[0, 1:].sum() >= n * 20
    # the last bin collects the long tracks
    _, _, sh2 = o.run(prim, n, np.arange(n), step_bins=8)
    assert np.array_equal(sh2[:, :7], sh[:, :7])
    assert np.array_equal(sh2[:, 7], sh[:, 7:].sum(1))


def test_field_crossing_of_a_cylinder(oracle_mod):
    """A 1 GeV e- leaves the origin along x in a 3.8 T field along z: the
    helix (radius p / (0.29979 B) m) meets r = 30 cm after the arc length
    2 r_h asin(30 / (2 r_h)); the step that crosses ends on the surface to
    within the RK4 miss distance and moves the track into the Si shell."""
    s = W.cms_field_setup()
    o = make(oracle_mod, s)
    T = 1000.0
    p = np.sqrt(T * (T + 2 * 0.51099895))
    rh = p / (2.99792458 * 3.8)
    arc = 2 * rh * np.arcsin(30.0 / (2 * rh))
    t = np.array([1, T, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0, 0], float)
    total = 0.0
    for _ in range(10):
        t, sec, info = o.step_one(t, 1, 0)
        total += info[0]
        if info[2]:
            break
    assert info[2] == 1 and t[8] == 1
    assert abs(total - arc) < 1e-4
    assert abs(np.hypot(t[2], t[3]) - 30.0) < 1e-4
    assert t[1] == T  # no loss in vacuum
