"""The pipelined schedule (one kernel per step: the interactions queued in
one iteration are sampled in the next, alongside that iteration's
transport) against the FP64 oracle and against the other schedules: only
the iteration in which an interacting track's step completes changes, so
every result is the same (up to the summation order of deposits)."""
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


def run(emt, s, prim, n, **kw):
    kw.setdefault("slot_capacity", 1 << 22)
    ids = np.arange(n, dtype=np.uint64)
    ctx = emt.context_for(s, max_events=n, **kw)
    ctx.submit(ids, prim)
    st = ctx.run()
    hist, summ, got = ctx.read_all()
    assert ctx.events_in_flight() == 0 and emt.lib().emt_tracks_in_flight(ctx._h) == 0
    ctx.close()
    assert np.array_equal(got, ids)
    return hist, summ, st


def same(a, b):
    (h1, s1, _), (h2, s2, _) = a, b
    assert np.array_equal(s1[:, 4:], s2[:, 4:])
    assert np.allclose(s1[:, :4], s2[:, :4], rtol=1e-12, atol=0)
    assert np.allclose(h1, h2, rtol=1e-12, atol=1e-12)


def against_oracle(oracle_mod, s, prim, n, hist, summ):
    ohist, osumm = oracle_of(oracle_mod, s).run(prim, n, np.arange(n))
    e_in = osumm[:, 3]
    rel = np.abs(summ[:, 0] - osumm[:, 0]) / e_in
    assert (rel <= TOL).mean() >= 0.999, np.sort(rel)[-3:]
    assert (np.abs(hist - ohist).max(axis=1) / e_in <= TOL).mean() >= 0.999
    same_counts = (summ[:, 4] == osumm[:, 4]) & (summ[:, 5] == osumm[:, 5])
    assert same_counts.mean() >= 0.999


@pytest.mark.parametrize("loop", ["plain", "graph"])
def test_pipelined_calo_matches_oracle(emt, oracle_mod, loop):
    s = W.calo_setup()
    n = 300
    prim = W.calo_primaries(n)
    hist, summ, st = run(emt, s, prim, n, schedule="pipelined", loop_mode=loop, graph_steps=24)
    against_oracle(oracle_mod, s, prim, n, hist, summ)
    ref = run(emt, s, prim, n, schedule="split", loop_mode="graph", graph_steps=24)
    assert st["track_steps"] == ref[2]["track_steps"]
    assert st["iterations"] > ref[2]["iterations"]  # an interacting step completes one iteration later


def test_pipelined_field_matches_oracle(emt, oracle_mod):
    s = W.calo_field_setup()
    n = 200
    prim = W.calo_field_primaries(n)
    hist, summ, st = run(emt, s, prim, n, schedule="pipelined", loop_mode="graph", graph_steps=24,
                         slot_capacity=1 << 23)
    against_oracle(oracle_mod, s, prim, n, hist, summ)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pipelined_equals_split_and_fused(emt, precision):
    s = W.calo_field_setup()
    n = 40
    prim = W.multi_primaries(n, 1, 6, 200.0, 20.0, seed=61)
    fused = run(emt, s, prim, n, precision=precision, schedule="fused")
    split = run(emt, s, prim, n, precision=precision, schedule="split")
    pipe = run(emt, s, prim, n, precision=precision, schedule="pipelined", loop_mode="graph", graph_steps=12)
    same(fused, pipe)
    same(split, pipe)


def test_pipelined_deferral_and_cylinders(emt):
    """A track store too small for the showers defers interactions (they
    wait in the queue), and the cylinder geometry; results unchanged."""
    s = W.calo_setup()
    n = 30
    prim = W.multi_primaries(n, 1, 6, 200.0, 20.0, seed=62)
    ref = run(emt, s, prim, n, schedule="fused")
    small = run(emt, s, prim, n, schedule="pipelined", slot_capacity=3000)
    assert small[2]["deferred"] > 0
    same(ref, small)
    c = W.cms_setup()
    cp = W.cms_primaries(6, 40, seed=63)
    same(run(emt, c, cp, 6, schedule="fused"), run(emt, c, cp, 6, schedule="pipelined"))


def test_pipelined_refuses_explicit_track_states(emt):
    s = W.calo_setup()
    ctx = emt.context_for(s, slot_capacity=1 << 12, max_events=2, schedule="pipelined")
    with pytest.raises(emt.EmtError) as e:
        ctx.debug_get_tracks()
    assert e.value.status == -4
    ctx.close()


@pytest.mark.parametrize("schedule,loop", [("split", "graph"), ("fused", "plain"), ("pipelined", "graph"),
                                           ("fused", "persistent")])
def test_slot_overflow_moves_tracks_to_host(emt, schedule, loop):
    """Showers far larger than the track store: when no track can take its
    next step, half of the stored tracks wait in host memory and come back
    later; every result equals the unlimited run's."""
    s = W.calo_setup()
    n = 24
    prim = W.calo_primaries(n, energy=10000.0, seed=64)
    ref = run(emt, s, prim, n, schedule="split", slot_capacity=1 << 22)
    small = run(emt, s, prim, n, schedule=schedule, loop_mode=loop, graph_steps=12, slot_capacity=512)
    assert ref[2]["peak_tracks"] > 16 * 512
    assert small[2]["spilled"] > 0 and small[2]["deferred"] > 0
    same(ref, small)
