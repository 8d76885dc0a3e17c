"""The persistent step loop (EMT_LOOP_PERSISTENT: one cooperative kernel
runs many steps with a grid barrier between them) gives the same results as
the host-driven loop, and its bounded barrier wait gives up with
EMT_ERR_TIMEOUT instead of hanging (made to run out on purpose by a
barrier that one participant never reaches; no GPU fault involved)."""
import time

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


def run(emt, s, prim, n, max_iterations=0, **kw):
    kw.setdefault("slot_capacity", 1 << 22)
    ids = np.arange(n, dtype=np.uint64)
    ctx = emt.context_for(s, max_events=n, **kw)
    ctx.submit(ids, prim)
    stats = []
    while True:
        st = ctx.run(max_iterations=max_iterations)
        stats.append(st)
        if st["live_tracks"] == 0:
            break
    hist, summ, got = ctx.read_all()
    ctx.close()
    assert np.array_equal(got, ids)
    return hist, summ, stats


def same(a, b):
    (h1, s1, _), (h2, s2, _) = a, b
    assert np.array_equal(s1[:, 4:], s2[:, 4:])
    assert np.allclose(s1[:, :4], s2[:, :4], rtol=1e-12, atol=0)
    assert np.allclose(h1, h2, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("setup,precision", [("calo", "fp64"), ("calo_field", "fp64"), ("calo_field", "mixed"),
                                             ("cms", "fp64")])
def test_persistent_loop_matches_host_loop(emt, setup, precision):
    if setup == "cms":
        s, prim, n = W.cms_setup(), W.cms_primaries(6, 40, seed=8), 6
    else:
        s = W.calo_setup() if setup == "calo" else W.calo_field_setup()
        n = 40
        prim = W.multi_primaries(n, 1, 5, 300.0, 20.0, seed=51)
    plain = run(emt, s, prim, n, precision=precision, loop_mode="plain", schedule="fused")
    pers = run(emt, s, prim, n, precision=precision, loop_mode="persistent", graph_steps=48)
    same(plain, pers)
    steps = sum(st["iterations"] for st in pers[2])
    launches = sum(st["kernel_launches"] for st in pers[2])
    assert launches < steps  # many steps per launch
    assert sum(st["track_steps"] for st in pers[2]) == int(plain[1][:, 4].sum())


def test_persistent_loop_partial_runs_and_deferral(emt):
    """Runs limited to a few iterations at a time, and a track store small
    enough to defer steps, give the same results."""
    s = W.calo_setup()
    n = 30
    prim = W.multi_primaries(n, 1, 6, 200.0, 20.0, seed=52)
    ref = run(emt, s, prim, n, loop_mode="plain", schedule="fused")
    part = run(emt, s, prim, n, max_iterations=7, loop_mode="persistent", graph_steps=64)
    same(ref, part)
    assert all(st["iterations"] <= 7 for st in part[2])
    small = run(emt, s, prim, n, loop_mode="persistent", graph_steps=32, slot_capacity=3000)
    assert sum(st["deferred"] for st in small[2]) > 0
    same(ref, small)


def test_bounded_wait_gives_up(emt):
    """A grid barrier that is never released: the wait runs out after its
    limit, the kernel ends, EMT_ERR_TIMEOUT is reported, and the GPU keeps
    working."""
    L = emt.lib()
    t0 = time.perf_counter()
    rc = L.emt_debug_wait_timeout(0, 200)
    dt = time.perf_counter() - t0
    assert rc == -5
    assert 0.15 < dt < 10.0
    s = W.calo_setup()
    prim = W.calo_primaries(4, energy=500.0)
    h, sm, _ = run(emt, s, prim, 4, loop_mode="persistent", graph_steps=48)
    led = np.abs(sm[:, 3] - sm[:, 0] - sm[:, 1] - sm[:, 2]) / sm[:, 3]
    assert led.max() < 1e-9 and sm[:, 4].min() > 0
