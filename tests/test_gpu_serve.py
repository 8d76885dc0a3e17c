"""Serving loop (emt_serve): requests arriving while others are on the GPU
are admitted as slots free up, and every event's result is the same as when
it runs alone (up to the summation order of FP64 deposits)."""
import numpy as np
import pytest

from paper_2203_09467_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emt():
    import torch
    assert torch.cuda.is_available()
    from paper_2203_09467_gb300 import emt as E
    E.lib()
    return E


def overlapping_admissions(admit, done):
    """Requests admitted while an earlier-admitted request was still on the
    GPU (admitted, not yet finished)."""
    n = 0
    for j in range(len(admit)):
        earlier = admit < admit[j]
        n += int(np.any(earlier & (done > admit[j])))
    return n


def alone(emt, s, prim, e, event_id, **kw):
    sub = W.subset(prim, [e])
    ctx = emt.context_for(s, slot_capacity=1 << 20, max_events=1, **kw)
    ctx.submit([event_id], sub)
    ctx.run()
    h, sm, _ = ctx.read_all()
    ctx.close()
    return h[0], sm[0]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_served_results_equal_alone(emt, precision):
    s = W.calo_field_setup()
    n = 60
    prim = W.multi_primaries(n, 1, 6, 500.0, 10.0, seed=31)
    ids = np.arange(5000, 5000 + n, dtype=np.uint64)
    arrival = np.sort(np.random.default_rng(3).uniform(0, 0.5, n))
    ctx = emt.context_for(s, slot_capacity=1 << 21, max_events=16, precision=precision, loop_mode="graph",
                          graph_steps=6)
    admit, done, hist, summ = ctx.serve(ids, arrival, prim, mode="continuous", steps_per_poll=6, time_scale=1.0)
    assert ctx.events_in_flight() == 0
    ctx.close()
    assert np.all(admit >= arrival - 1e-3) and np.all(done >= admit)
    # continuous batching: requests were admitted while others were in flight
    assert overlapping_admissions(admit, done) > 0
    # the ledger closes on every event (FP64 exactly; mixed to FP32 rounding)
    led = np.abs(summ[:, 3] - summ[:, 0] - summ[:, 1] - summ[:, 2]) / summ[:, 3]
    assert led.max() < (1e-9 if precision == "fp64" else 1e-5)
    for e in (0, 17, 41, 59):
        h1, s1 = alone(emt, s, prim, e, ids[e], precision=precision)
        assert np.array_equal(s1[4:], summ[e, 4:])
        assert np.allclose(s1[:4], summ[e, :4], rtol=1e-12, atol=0)
        assert np.allclose(h1, hist[e], rtol=1e-12, atol=1e-12)


def test_batch_schedule_matches_continuous(emt):
    s = W.calo_setup()
    n = 40
    prim = W.multi_primaries(n, 1, 4, 300.0, 10.0, seed=32)
    ids = np.arange(n, dtype=np.uint64)
    arrival = np.linspace(0, 0.2, n)
    out = {}
    for mode in ("continuous", "batch"):
        ctx = emt.context_for(s, slot_capacity=1 << 21, max_events=8)
        out[mode] = ctx.serve(ids, arrival, prim, mode=mode, steps_per_poll=4)
        ctx.close()
    # one batch at a time: nothing is admitted while an earlier batch runs;
    # continuously: requests join the events in flight
    assert overlapping_admissions(out["batch"][0], out["batch"][1]) == 0
    assert overlapping_admissions(out["continuous"][0], out["continuous"][1]) > 0
    assert np.array_equal(out["continuous"][3][:, 4:], out["batch"][3][:, 4:])
    assert np.allclose(out["continuous"][3][:, :4], out["batch"][3][:, :4], rtol=1e-12, atol=0)
