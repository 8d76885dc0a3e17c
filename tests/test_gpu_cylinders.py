"""The concentric-cylinder geometry of the paper's Sec. 3.2 test problem on
the GPU (through the C ABI) against the FP64 oracle: single steps from
random states in every shell, whole events (straight and in a solenoid
field, both step schedules), deposition scored along z, the
steps-per-track histogram and the per-step trace.

Tolerances as in test_gpu_parity: the FP64 path repeats the oracle's
arithmetic in the same order, so positions agree to rounding, step and
track counts exactly, deposits (totals and every bin) to 1e-9 of the event
energy (summation order of the atomics), in the field too."""
import numpy as np
import pytest

from paper_2203_09467_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def emt():
    import torch
    assert torch.cuda.is_available()
    from paper_2203_09467_gb300 import emt as E
    E.lib()
    return E


def oracle_of(oracle_mod, s):
    return oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)


def gpu_run(emt, s, prim, n_events, **kw):
    ids = np.arange(n_events, dtype=np.uint64)
    kw.setdefault("slot_capacity", 1 << 22)
    kw.setdefault("max_events", max(n_events, 1))
    ctx = emt.context_for(s, **kw)
    ctx.submit(ids, prim)
    st = ctx.run()
    hist, summ, got = ctx.read_all()
    sh = ctx.read_step_hist() if kw.get("step_hist_bins") else None
    ctx.close()
    assert np.array_equal(got, ids)
    return hist, summ, st, sh


def check_events(summ, osumm, hist, ohist, frac=1.0, bin_tol=TOL):
    e_in = osumm[:, 3]
    assert np.allclose(summ[:, 3], e_in, rtol=1e-13, atol=0)
    rel = np.abs(summ[:, 0] - osumm[:, 0]) / e_in
    assert (rel <= TOL).mean() >= frac, np.sort(rel)[-3:]
    same = (summ[:, 4] == osumm[:, 4]) & (summ[:, 5] == osumm[:, 5])
    assert same.mean() >= frac
    led = np.abs(summ[:, 3] - summ[:, 0] - summ[:, 1] - summ[:, 2]) / summ[:, 3]
    assert led.max() <= TOL
    hrel = np.abs(hist - ohist).max(axis=1) / e_in
    assert (hrel <= bin_tol).mean() >= frac, np.sort(hrel)[-3:]


def test_single_step_parity_cylinders(emt, oracle_mod):
    """Random states in every shell (all particle types, energies from 1 MeV
    to 30 GeV, isotropic directions), one step each on the GPU and in the
    oracle: survivors and secondaries agree in type, volume, step count,
    energy, position and direction."""
    s = W.cms_setup()
    rng = np.random.default_rng(21)
    n = 3000
    R = (0.0,) + W.CMS_RADII
    rec = np.zeros((n, 10))
    rec[:, 0] = rng.integers(0, 3, n)
    rec[:, 1] = 10 ** rng.uniform(0.05, 4.5, n)
    vol = rng.integers(0, 6, n)
    r = np.sqrt(rng.uniform(np.take(R, vol) ** 2, np.take(R, vol + 1) ** 2))
    phi = rng.uniform(0, 2 * np.pi, n)
    rec[:, 2], rec[:, 3] = r * np.cos(phi), r * np.sin(phi)
    rec[:, 4] = rng.uniform(-W.CMS_HALF_Z, W.CMS_HALF_Z, n)
    rec[:, 8] = vol
    d = rng.normal(size=(n, 3))
    rec[:, 5:8] = d / np.linalg.norm(d, axis=1, keepdims=True)
    rec[:, 9] = rng.integers(0, 50, n)
    uid = rng.integers(1, 2 ** 63, n, dtype=np.uint64)
    n_ev = 16
    ev_ids = rng.integers(0, 2 ** 40, n_ev, dtype=np.uint64)
    slot = rng.integers(0, n_ev, n)
    ctx = emt.context_for(s, slot_capacity=1 << 16, max_events=n_ev)
    empty = {"event": np.zeros(0, np.int32), "type": np.zeros(0, np.int32), "T": np.zeros(0),
             "pos": np.zeros((0, 3)), "dir": np.zeros((0, 3))}
    ctx.submit(ev_ids, empty)
    ctx.debug_set_tracks(rec, uid, slot.astype(np.int32))
    ctx.run(max_iterations=1)
    grec, guid, _ = ctx.debug_get_tracks()
    o = oracle_of(oracle_mod, s)
    want = {}
    for i in range(n):
        t, sec, info, suid = o.step_one(rec[i], int(uid[i]), int(ev_ids[slot[i]]), with_uids=True)
        if info[5]:
            want[int(uid[i])] = t
        for k in range(len(sec)):
            want[int(suid[k])] = np.array([*sec[k][:8], t[8], 0.0])
    got = {int(u): r for u, r in zip(guid, grec)}
    assert set(got) == set(want)
    bad = [(got[u], want[u]) for u in want
           if got[u][0] != want[u][0] or got[u][8] != want[u][8] or got[u][9] != want[u][9]
           or not np.allclose(got[u][1:8], want[u][1:8], rtol=1e-11, atol=1e-11)]
    assert not bad, bad[:3]
    ctx.debug_set_tracks(np.zeros((0, 10)), np.zeros(0, np.uint64), np.zeros(0, np.int32))
    ctx.read_all()
    ctx.close()


@pytest.mark.parametrize("schedule", ["fused", "split"])
def test_cms_event_parity(emt, oracle_mod, schedule):
    """Sec. 3.2's problem at reduced size (12 events x 50 photons of 1 GeV):
    z profile, totals, step and track counts and the steps-per-track
    histogram by particle type all match the oracle."""
    s = W.cms_setup()
    n = 12
    prim = W.cms_primaries(n, 50)
    nb = 4096
    hist, summ, st, sh = gpu_run(emt, s, prim, n, schedule=schedule, step_hist_bins=nb)
    ohist, osumm, osh = oracle_of(oracle_mod, s).run(prim, n, np.arange(n), step_bins=nb)
    check_events(summ, osumm, hist, ohist)
    assert np.array_equal(sh, osh)
    assert st["track_steps"] == int(osumm[:, 4].sum())


def test_cms_full_size(emt, oracle_mod):
    """Sec. 3.2's problem at its full size (100 events x 1000 isotropic
    photons of 1 GeV, 8.0e7 track-steps), in the benchmark's launch
    configuration (split schedule, graphs of 12 steps, 2^25 slots): every
    event, its z profile and the steps-per-track histogram match the
    oracle (about 1 s on 16 cores)."""
    s = W.cms_setup()
    n = 100
    prim = W.cms_primaries(n, 1000)
    nb = 4096
    hist, summ, st, sh = gpu_run(emt, s, prim, n, schedule="split", loop_mode="graph", graph_steps=12,
                                 slot_capacity=1 << 25, step_hist_bins=nb)
    ohist, osumm, osh = oracle_of(oracle_mod, s).run(prim, n, np.arange(n), step_bins=nb)
    check_events(summ, osumm, hist, ohist)
    assert np.array_equal(sh, osh)
    assert st["track_steps"] == int(osumm[:, 4].sum())


def test_cms_field_parity(emt, oracle_mod):
    s = W.cms_field_setup()
    n = 8
    prim = W.cms_primaries(n, 25, seed=9)
    hist, summ, st, _ = gpu_run(emt, s, prim, n, schedule="split")
    ohist, osumm = oracle_of(oracle_mod, s).run(prim, n, np.arange(n))
    check_events(summ, osumm, hist, ohist)


def test_layers_scored_along_z(emt, oracle_mod):
    """Scoring along z on the layered calorimeter: 70 bins of 5 mm."""
    s = W.calo_setup()
    s.world = W.world(0.0, 20.0, 20.0, (-100.0, -100.0, -50.0), (100.0, 100.0, 85.0), n_bins=70,
                      score_z=(0.0, 35.0))
    n = 40
    prim = W.calo_primaries(n, energy=3000.0)
    hist, summ, st, _ = gpu_run(emt, s, prim, n, schedule="split")
    ohist, osumm = oracle_of(oracle_mod, s).run(prim, n, np.arange(n))
    check_events(summ, osumm, hist, ohist)


def test_step_trace(emt):
    """Per-step records of the paper's Fig. "tracks in flight": the first
    step of photons born in the vacuum core is all boundary crossings, the
    records account for every track-step and deferred copy, and the
    per-step device times add up to the run's kernel time."""
    s = W.cms_setup()
    n = 20
    prim = W.cms_primaries(n, 100)
    ctx = emt.context_for(s, slot_capacity=1 << 22, max_events=n, schedule="split", loop_mode="graph",
                          graph_steps=12)
    ctx.submit(np.arange(n, dtype=np.uint64), prim)
    st, rec = ctx.run_traced()
    ctx.read_all()
    ctx.close()
    assert len(rec) == st["iterations"]
    assert rec[0, 0] == n * 100 and rec[0, 1] == 0 and rec[0, 2] == 0
    assert rec[1, 0] > 0 and rec[1, 2] > 0  # the photons reach the silicon
    assert (rec[:, 0] + rec[:, 1]).sum() == st["track_steps"] + st["deferred"]
    assert rec[:, 3].sum() == st["deferred"]
    assert rec[:, 4].sum() == st["held"] == 0
    assert abs(rec[:, 5].sum() - st["kernel_ms"]) <= 1e-6 * st["kernel_ms"] + 1e-3
    assert (rec[:, 5] > 0).all()


def test_cms_mixed_statistical(emt, oracle_mod):
    """Mixed precision on Sec. 3.2's problem: totals, the z profile (Hotelling
    T^2 over groups of bins) and the mean steps per track of each particle
    type agree with the FP64 oracle within their statistical errors."""
    from stats_util import profile_test, mean_test
    s = W.cms_setup(n_bins=70)
    n = 400
    prim = W.cms_primaries(n, 10, seed=12)
    nb = 4096
    hist, summ, st, sh = gpu_run(emt, s, prim, n, precision="mixed", schedule="split", step_hist_bins=nb)
    ohist, osumm, osh = oracle_of(oracle_mod, s).run(prim, n, np.arange(n), step_bins=nb)
    led = np.abs(summ[:, 3] - summ[:, 0] - summ[:, 1] - summ[:, 2]) / summ[:, 3]
    assert led.max() < 1e-5
    d, se = mean_test(summ[:, 0], osumm[:, 0])
    assert abs(d) < 4 * se + 1e-6 * osumm[:, 0].mean()
    t2, dof, p = profile_test(hist, ohist)
    assert p > 0.01, (t2, dof, p)
    steps = np.arange(nb)
    for k in range(3):
        m_gpu = (sh[k] * steps).sum() / sh[k].sum()
        m_orc = (osh[k] * steps).sum() / osh[k].sum()
        assert abs(m_gpu / m_orc - 1) < 0.03, (k, m_gpu, m_orc)


def test_cylinder_edge_cases(emt, oracle_mod):
    """Primaries outside the envelope (beyond r = 375 cm, beyond the end
    planes), below the cut, on the axis moving along z (no radial surface
    ahead), exactly on a shell radius and on an end plane, in the vacuum
    core and in every material; compared event by event with the oracle."""
    s = W.cms_setup()
    R = W.CMS_RADII
    pos = [[0, 0, 0], [400.0, 0, 0], [0, 0, 701.0], [50.0, 0, 10.0], [0, 0, -3.0], [R[0], 0, 0],
           [0, -R[2], 20.0], [10.0, 0, 700.0], [200.0, 0, -650.0], [340.0, 10.0, 0]]
    dirs = [[1, 0, 0], [1, 0, 0], [0, 0, 1], [0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1],
            [0.6, 0, -0.8], [-1, 0, 0]]
    types = [0, 1, 0, 2, 0, 1, 2, 0, 1, 0]
    T = [1000.0, 500.0, 300.0, 0.6, 2000.0, 800.0, 3000.0, 50.0, 400.0, 700.0]
    n = len(pos)
    prim = {"event": np.arange(n, dtype=np.int32), "type": np.array(types, np.int32), "T": np.array(T),
            "pos": np.array(pos, float), "dir": np.array(dirs, float)}
    hist, summ, st, _ = gpu_run(emt, s, prim, n)
    ohist, osumm = oracle_of(oracle_mod, s).run(prim, n, np.arange(n))
    assert summ[1, 1] == 500.0 and summ[2, 1] == 300.0   # outside the world: escaped
    assert summ[3, 0] == 0.6 + 2 * 0.51099895 or abs(summ[3, 0] - (0.6 + 2 * 0.51099895)) < 1e-12
    check_events(summ, osumm, hist, ohist)


def test_invalid_geometry_and_options_rejected(emt):
    """Cylinders need z0 = 0 and a positive half-length; scoring along z needs
    a non-empty range; track selection needs the split schedule, the host
    spill low-energy selection with a budget at least max_active."""
    s = W.cms_setup()
    ctx = emt.Context(slot_capacity=1 << 12, max_events=4, max_bins=200)
    ctx.load_materials(s.materials, s.physics)
    for k, v in [(0, 5.0), (17, 0.0), (20, -700.0)]:  # z0, half_z, score range
        w = s.world.copy()
        w[k] = v
        with pytest.raises(emt.EmtError) as e:
            ctx.load_geometry(s.layers, w)
        assert e.value.status == -1
    ctx.load_geometry(s.layers, s.world)
    ctx.close()
    for kw in [dict(max_active=100, schedule="fused"),
               dict(max_active=100, schedule="split", select="order", spill_above=200),
               dict(max_active=100, schedule="split", select="low_energy", spill_above=50)]:
        with pytest.raises(emt.EmtError):
            emt.Context(slot_capacity=1 << 12, max_events=4, **kw)
