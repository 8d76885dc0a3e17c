"""Mixed-precision path (FP32 tables, sampling and kinematics; FP64
positions, boundary distances and energy tallies) against the FP64 oracle.

The mixed path draws FP32 uniforms from the same counter-based streams, so
its showers are independent samples of the same physics: results are
compared statistically, and its error against the oracle is stated per
result (total deposition and per-layer profile).
"""
import numpy as np
import pytest
from paper_2203_09467_gb300 import workloads as W
from stats_util import profile_test

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emt():
    import torch
    assert torch.cuda.is_available()
    from paper_2203_09467_gb300 import emt as E
    E.lib()
    return E


def run(emt, s, prim, n, precision):
    ctx = emt.context_for(s, slot_capacity=1 << 24, max_events=n, precision=precision)
    ctx.submit(np.arange(n, dtype=np.uint64), prim)
    st = ctx.run()
    hist, summ, _ = ctx.read_all()
    ctx.close()
    return hist, summ, st


@pytest.mark.parametrize("workload", ["calo", "calo_field"])
def test_mixed_matches_oracle_statistically(emt, oracle_mod, workload):
    if workload == "calo":
        s = W.calo_setup()
        n = 1500
        prim = W.calo_primaries(n, energy=2000.0)
    else:
        s = W.calo_field_setup()
        n = 600
        prim = W.calo_field_primaries(n, e_min=200.0, e_ratio=20.0)
    hm, sm, st = run(emt, s, prim, n, "mixed")
    o = oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
    ho, so = o.run(prim, n, np.arange(n))
    # energy ledger: FP32 kinematics conserve energy to FP32 rounding per interaction
    led = np.abs(sm[:, 3] - sm[:, 0] - sm[:, 1] - sm[:, 2]) / sm[:, 3]
    assert led.max() < 1e-5, led.max()
    # total deposition: difference of means within 4 standard errors
    d = sm[:, 0].mean() - so[:, 0].mean()
    se = np.sqrt(sm[:, 0].var(ddof=1) / n + so[:, 0].var(ddof=1) / n)
    assert abs(d) < 4 * se + 1e-6 * so[:, 0].mean(), (d, se)
    # longitudinal profile
    t2, dof, p = profile_test(hm, ho)
    assert p > 0.01, (t2, dof, p)
    # steps per event agree to within a few percent on average
    assert abs(sm[:, 4].mean() / so[:, 4].mean() - 1) < 0.03


def test_mixed_error_statement(emt, oracle_mod):
    """The mixed path's error against the FP64 oracle, per result, on 4,000
    events of 10 GeV electrons in the calorimeter (independent samples):
    total deposition (difference of means and its standard error), the
    sampling fraction in LAr, the per-layer profile (Hotelling T^2) and the
    worst per-event energy ledger.  Printed for the record; the asserts are
    the statistical bars of the test above."""
    from stats_util import mean_test
    s = W.calo_setup()
    n = 4000
    prim = W.calo_primaries(n)
    hm, sm, _ = run(emt, s, prim, n, "mixed")
    o = oracle_mod.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
    ho, so = o.run(prim, n, np.arange(n))
    d, se = mean_test(sm[:, 0], so[:, 0])
    fm = hm[:, 1::2].sum(1) / hm.sum(1)
    fo = ho[:, 1::2].sum(1) / ho.sum(1)
    dfr, sefr = mean_test(fm, fo)
    t2, dof, p = profile_test(hm, ho)
    led = np.abs(sm[:, 3] - sm[:, 0] - sm[:, 1] - sm[:, 2]) / sm[:, 3]
    print(f"\nmixed vs FP64 oracle, {n} x 10 GeV e-: total deposition {sm[:, 0].mean():.3f} vs "
          f"{so[:, 0].mean():.3f} MeV, difference {d:+.3f} +- {se:.3f} MeV ({d / se:+.2f} sigma); "
          f"LAr sampling fraction {fm.mean():.5f} vs {fo.mean():.5f} ({dfr / sefr:+.2f} sigma); "
          f"profile T2 = {t2:.1f} on {dof} groups, p = {p:.3f}; worst ledger {led.max():.2e}; "
          f"steps/event {sm[:, 4].mean():.0f} vs {so[:, 4].mean():.0f}")
    assert abs(d) < 4 * se + 1e-6 * so[:, 0].mean()
    assert abs(dfr) < 4 * sefr
    assert p > 0.01
    assert led.max() < 1e-5


def test_mixed_is_deterministic(emt):
    s = W.calo_setup()
    prim = W.calo_primaries(200, energy=3000.0)
    h1, s1, _ = run(emt, s, prim, 200, "mixed")
    h2, s2, _ = run(emt, s, prim, 200, "mixed")
    assert np.array_equal(s1[:, 4:], s2[:, 4:])
    assert np.allclose(s1[:, :4], s2[:, :4], rtol=1e-12, atol=0)
