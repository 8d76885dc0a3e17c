"""Pins of the oracle's transport loop: geometry by brute-force counting,
exponential free paths, continuous slowing down against the range table,
slab transmission against exp(-Sigma L), RK4 against the analytic helix,
and the per-event energy ledger."""
import numpy as np
import pytest
from scipy import stats

from paper_2203_09467_gb300 import workloads as W

ME = 0.51099895


def make(oracle_mod, s):
    return oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)


def one_primary(t, T, pos, d):
    return {"event": np.array([0], np.int32), "type": np.array([t], np.int32),
            "T": np.array([T]), "pos": np.array([pos], float), "dir": np.array([d], float)}


def test_straight_photon_crosses_every_layer(oracle_mod):
    s = W.calo_setup(mask=0)
    o = make(oracle_mod, s)
    hist, summ = o.run(one_primary(0, 50.0, [0, 0, -1], [0, 0, 1]), 1, [0])
    # enter the stack, 100 layers, leave the world
    assert summ[0, 4] == 102 and summ[0, 1] == 50.0 and summ[0, 0] == 0.0
    # boundary positions are exactly the planes
    t = np.array([0, 50.0, 0.3, -0.2, -1.0, 0, 0, 1, -1, 0], float)
    zs = []
    for _ in range(101):
        t, sec, info = o.step_one(t, 1, 0)
        zs.append(t[4])
        assert info[2] == 1
    planes = np.concatenate([[0.0], np.cumsum(s.layers[:, 1])])
    assert zs == list(planes)


@pytest.mark.parametrize("deg", [5.0, 30.0, 60.0, 85.0])
def test_oblique_photon_layer_count(oracle_mod, deg):
    s = W.calo_setup(mask=0)
    o = make(oracle_mod, s)
    th = np.deg2rad(deg)
    d = [np.sin(th), 0.0, np.cos(th)]
    hist, summ = o.run(one_primary(0, 50.0, [0, 0, -1], d), 1, [0])
    planes = np.concatenate([[0.0], np.cumsum(s.layers[:, 1])])
    x_at = lambda z: (z + 1.0) * np.tan(th)
    # brute force: walk the planes; the photon leaves through x = 20 at z_side
    z_side = -1.0 + 20.0 / np.tan(th)
    visited = 1 + int(np.sum(planes[1:-1] < z_side))
    steps = 1 + visited + 1
    assert x_at(0.0) < 20.0
    assert summ[0, 4] == steps


def test_free_path_is_exponential(oracle_mod):
    s = W.slab_setup(mask=2, thickness=1e4)  # Compton only
    s.world[3:9] = [-1e5, -1e5, -1e5, 1e5, 1e5, 1e5]
    s.world[1] = s.world[2] = 1e4
    o = make(oracle_mod, s)
    grid = o.grid()
    k = grid[40]
    sigma = o.table(0, 0, 1)[40]
    lengths = []
    for uid in range(1, 20001):
        t = np.array([0, k, 0, 0, 5e3, 0, 0, 1, 0, 0], float)
        t, sec, info = o.step_one(t, uid, 3)
        assert info[3] == 1
        lengths.append(info[0])
    lengths = np.array(lengths)
    assert stats.kstest(lengths * sigma, "expon").pvalue > 1e-3
    assert abs(lengths.mean() * sigma - 1) < 4 / np.sqrt(len(lengths))


def test_continuous_slowing_down_follows_range(oracle_mod):
    s = W.slab_setup(mask=0, thickness=100.0)
    s.world[1] = s.world[2] = 100.0
    o = make(oracle_mod, s)
    T0 = 500.0
    t = np.array([1, T0, 0, 0, 1.0, 0, 0, 1, 0, 0], float)
    path, edep = 0.0, 0.0
    R0 = o.range(0, 1, T0)
    for _ in range(1000):
        Tb = t[1]
        Rb = o.range(0, 1, Tb)
        t, sec, info = o.step_one(t, 1, 0)
        path += info[0]
        edep += info[1]
        # no discrete process and no boundary: every step is the e+- step
        # limit max(f R, min(R, r_final)) itself
        assert info[0] == pytest.approx(max(0.2 * Rb, min(Rb, 0.1)), rel=1e-12, abs=0)
        if info[5] == 0:
            break
    assert info[5] == 0
    assert abs(edep / T0 - 1) < 1e-12
    # the track stops when it falls below the cut: path = R(T0) - R(T_end)
    Tend = t[1]
    assert Tend < 1.0
    assert abs(path - (R0 - o.range(0, 1, Tend))) < 1e-9 * R0


def test_photoelectric_slab_transmission(oracle_mod):
    """Photo-only beam through a Pb slab: interacting fraction
    1 - exp(-Sigma L) (binomial), every interaction deposits k locally."""
    thick = 5.0
    s = W.slab_setup(mask=1, thickness=thick)
    s.physics[1] = s.physics[2] = 1e4  # electron cut above k: photoelectron deposits
    o = make(oracle_mod, s)
    grid = o.grid()
    k = grid[26]
    sigma = o.table(0, 0, 0)[26]
    n = 20000
    prim = {"event": np.arange(n, dtype=np.int32), "type": np.zeros(n, np.int32),
            "T": np.full(n, k), "pos": np.tile([0, 0, -1.0], (n, 1)),
            "dir": np.tile([0, 0, 1.0], (n, 1))}
    hist, summ = o.run(prim, n, np.arange(n))
    hit = summ[:, 0] > 0
    assert np.all(np.isclose(summ[hit, 0], k, rtol=1e-14))
    p = 1 - np.exp(-sigma * thick)
    assert abs(hit.mean() - p) < 4 * np.sqrt(p * (1 - p) / n)


def _ledger(summ):
    return np.abs(summ[:, 3] - summ[:, 0] - summ[:, 1] - summ[:, 2]) / summ[:, 3]


def test_energy_ledger_every_event(oracle_mod):
    s = W.slab_setup()
    o = make(oracle_mod, s)
    n = 1000
    hist, summ = o.run(W.slab_primaries(n), n, np.arange(n))
    assert _ledger(summ).max() < 1e-9
    assert np.allclose(hist[:, 0], summ[:, 0], rtol=1e-12)
    c = W.calo_setup()
    oc = make(oracle_mod, c)
    n = 100
    hist, summ = oc.run(W.calo_primaries(n), n, np.arange(n))
    assert _ledger(summ).max() < 1e-9
    assert np.allclose(hist.sum(1), summ[:, 0], rtol=1e-12)


def test_results_do_not_depend_on_thread_count(oracle_mod):
    c = W.calo_setup()
    o = make(oracle_mod, c)
    p = W.calo_primaries(24)
    h1, s1 = o.run(p, 24, np.arange(24), n_threads=1)
    h8, s8 = o.run(p, 24, np.arange(24), n_threads=8)
    assert np.array_equal(h1, h8) and np.array_equal(s1, s8)


def field_world(B=(2.0, 0, 0), half=1e3):
    s = W.slab_setup(mask=0, thickness=1.0)
    s.world[0] = 900.0                      # stack far away
    s.world[3:9] = [-half, -half, -half, half, half, half]
    s.world[9:12] = B
    s.world[15] = 5.0                      # max field step, cm
    return s


@pytest.mark.parametrize("pitch", [0.0, 0.3])
@pytest.mark.parametrize("T", [2.0, 50.0])
def test_rk4_matches_helix(oracle_mod, pitch, T):
    s = field_world()
    o = make(oracle_mod, s)
    u0 = np.array([pitch, np.sqrt(1 - pitch ** 2), 0.0])
    t = np.array([1, T, 0, 0, 0, *u0, -1, 0], float)
    p = np.sqrt(T * (T + 2 * ME))
    B = 2.0
    # each step is at most 100 substeps of h_max = sqrt(8 r delta) and at
    # most max_field_step; follow the helix over several steps to 5 cm
    hmax = np.sqrt(8 * (p / (2.99792458 * B)) * s.world[12])
    L = 0.0
    while L < 5.0 - 1e-9:
        t, sec, info = o.step_one(t, 1, 0)
        assert info[2] == 0 and info[3] == 0
        assert abs(info[0] - min(s.world[15], 100 * hmax)) < 1e-12
        L += info[0]
    q = -1.0
    # analytic helix about x: omega = q c B / p per unit path
    w = q * 2.99792458 * B / p
    ut = np.sqrt(1 - pitch ** 2)
    # du/ds = w u x B_hat, B_hat = x: (uy, uz)' = w (uz, -uy)
    uy = ut * np.cos(w * L)
    uz = -ut * np.sin(w * L)
    y = ut / w * np.sin(w * L)
    z = ut / w * (np.cos(w * L) - 1)
    want_x = np.array([pitch * L, y, z])
    assert np.linalg.norm(t[2:5] - want_x) < 1e-4
    assert np.linalg.norm(t[5:8] - [pitch, uy, uz]) < 1e-5
    assert abs(np.linalg.norm(t[5:8]) - 1) < 1e-14


def test_rk4_plane_crossing(oracle_mod):
    """An electron circling in vacuum hits the stack face z = z0: the step
    ends exactly on the plane after the analytic arc length (within the
    miss distance)."""
    s = field_world()
    s.world[0] = 1.0  # stack front face at z = 1
    o = make(oracle_mod, s)
    T = 50.0
    p = np.sqrt(T * (T + 2 * ME))
    w = -2.99792458 * 2.0 / p
    r = 1 / abs(w)
    t = np.array([1, T, 0, 0, 0, 0, 0, 1, -1, 0], float)  # moving +z, circling in y-z
    t, sec, info = o.step_one(t, 1, 0)
    assert info[2] == 1 and t[4] == 1.0 and t[8] == 0
    # circle through the origin tangent to +z: z(s) = r sin(s/r); z = 1
    s_exact = r * np.arcsin(1.0 / r)
    assert abs(info[0] - s_exact) < 1e-4


def test_shower_maximum_is_plausible(oracle_mod):
    """Loose physics sanity (not a parity pin): the longitudinal maximum of
    10 GeV showers in the Pb/LAr stack lies a few radiation lengths deep."""
    c = W.calo_setup()
    o = make(oracle_mod, c)
    n = 40
    hist, summ = o.run(W.calo_primaries(n), n, np.arange(n))
    prof = hist.mean(0)
    pair = prof[0::2] + prof[1::2]
    x0_pair = 0.2 / 0.5612 + 0.5 / 14.0
    tmax = (np.argmax(pair) + 0.5) * x0_pair
    assert 3.0 < tmax < 9.0
    assert 0.95 < summ[:, 0].mean() / 1e4 <= 1.0


@pytest.mark.parametrize("ptype,mask,node", [(0, 7, 40), (0, 7, 32), (1, 24, 40), (2, 56, 40), (2, 56, 28)])
def test_process_selection_frequencies(oracle_mod, ptype, mask, node):
    """The model of an interaction is chosen with probability Sigma_i /
    Sigma_tot (competing processes, Sec. 2.2): at a grid node the
    interpolated Sigma's are the table entries, so the counts over many
    independent draw streams are multinomial with those probabilities."""
    s = W.slab_setup(mask=mask, thickness=1e4)
    s.world[3:9] = [-1e5, -1e5, -1e5, 1e5, 1e5, 1e5]
    s.world[1] = s.world[2] = 1e4
    o = make(oracle_mod, s)
    T = o.grid()[node]
    nq = 3 if ptype != 1 else 2
    sig = np.array([o.table(0, ptype, q)[node] for q in range(nq)])
    pid_of = {0: [oracle_mod.PHOTO, oracle_mod.COMPTON, oracle_mod.PAIR],
              1: [oracle_mod.IONI, oracle_mod.BREMS],
              2: [oracle_mod.IONI, oracle_mod.BREMS, oracle_mod.ANNIH]}[ptype]
    counts = np.zeros(nq)
    n = 0
    for uid in range(1, 40001):
        t = np.array([ptype, T, 0, 0, 5e3, 0, 0, 1, 0, 0], float)
        t, sec, info = o.step_one(t, uid, 5)
        if info[3] != 1:
            continue  # an e+- step ended by its step limit
        counts[pid_of.index(int(info[4]))] += 1
        n += 1
    assert n > 5000
    expected = n * sig / sig.sum()
    keep = expected > 5
    assert stats.chisquare(counts[keep], expected[keep] * counts[keep].sum() / expected[keep].sum()).pvalue > 1e-3
    assert counts[~keep].sum() <= 3 * max(expected[~keep].sum(), 1.0)


def test_step_count_limit_kills_the_track(oracle_mod):
    """At the step limit the track ends and its energy (+ 2 m for e+) is
    tallied as killed; the ledger still closes."""
    for ptype, rest in [(1, 0.0), (2, 2 * ME)]:
        s = W.slab_setup(mask=0, thickness=100.0)
        s.world[1] = s.world[2] = 100.0
        s.world[13] = 3
        o = make(oracle_mod, s)
        T0 = 500.0
        t = np.array([ptype, T0, 0, 0, 1.0, 0, 0, 1, 0, 0], float)
        for _ in range(3):
            t, sec, info = o.step_one(t, 1, 0)
        assert info[5] == 0 and info[7] == pytest.approx(t[1] + rest, rel=1e-15)
        hist, summ = o.run(one_primary(ptype, T0, [0, 0, 1.0], [0, 0, 1]), 1, [0])
        assert summ[0, 4] == 3 and summ[0, 5] == 1
        assert summ[0, 2] == pytest.approx(t[1] + rest, rel=1e-12)
        assert summ[0, 0] + summ[0, 2] == pytest.approx(T0 + rest, rel=1e-12)


def test_deposits_are_scored_in_the_volume_traversed(oracle_mod):
    """A step's continuous loss is scored in the bin of the volume the step
    was taken in (the pre-step volume), also when the step ends on a plane:
    the histogram of a full run equals the per-step deposits binned by the
    pre-step layer."""
    s = W.calo_setup(mask=0)
    o = make(oracle_mod, s)
    T0 = 300.0
    t = np.array([1, T0, 0.1, 0.2, -1.0, 0, 0, 1, -1, 0], float)
    expected = np.zeros(o.n_bins)
    crossings = 0
    for _ in range(100000):
        vol = int(t[8])
        t, sec, info = o.step_one(t, 1, 0)
        if info[1] != 0.0:
            assert vol >= 0
            expected[int(s.layers[vol, 2])] += info[1]
        crossings += int(info[2])
        if info[5] == 0:
            break
    assert info[5] == 0 and crossings > 10
    hist, summ = o.run(one_primary(1, T0, [0.1, 0.2, -1.0], [0, 0, 1]), 1, [0])
    assert np.count_nonzero(expected) > 10
    np.testing.assert_allclose(hist[0, : o.n_bins], expected, rtol=1e-12, atol=0)


def test_closed_channel_is_a_null_interaction(oracle_mod):
    """Between the node below the pair threshold (Sigma = 0) and the one above
    it, the interpolated Sigma_pair is positive below 2 m: the photon can
    choose pair production where the channel is closed, and the step is
    then a null interaction (the photon goes on unchanged, nothing is
    deposited or produced, the step is counted)."""
    s = W.slab_setup(mask=4, thickness=1e4)
    s.world[3:9] = [-1e5, -1e5, -1e5, 1e5, 1e5, 1e5]
    s.world[1] = s.world[2] = 1e4
    o = make(oracle_mod, s)
    g = o.grid()
    n = int(np.searchsorted(g, 2 * ME))
    assert o.table(0, 0, 2)[n - 1] == 0.0 and o.table(0, 0, 2)[n] > 0.0
    T = 0.5 * (max(g[n - 1], s.physics[0]) + 2 * ME)
    for uid in range(1, 201):
        t0 = np.array([0, T, 0, 0, 5e3, 0, 0, 1, 0, 0], float)
        t, sec, info = o.step_one(t0.copy(), uid, 3)
        assert info[3] == 1 and int(info[4]) == oracle_mod.PAIR and info[5] == 1
        assert len(sec) == 0 and info[1] == 0.0
        assert t[1] == T and list(t[5:8]) == [0, 0, 1] and t[9] == 1
        assert t[4] == pytest.approx(5e3 + info[0], rel=1e-15)
