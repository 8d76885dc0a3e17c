"""The seeded input generators follow the recipe the workloads state: beam
spot, energies, particle mix, cone and isotropic directions, event sizes,
Poisson arrivals (no GPU needed)."""
import numpy as np
from scipy import stats

from paper_2203_09467_gb300 import workloads as W


def _unit(d):
    return np.allclose(np.linalg.norm(d, axis=1), 1.0, rtol=0, atol=1e-15)


def test_calorimeter_beam():
    p = W.calo_primaries()
    assert len(p["T"]) == 10000 and np.array_equal(p["event"], np.arange(10000))
    assert np.all(p["type"] == W.ELECTRON) and np.all(p["T"] == 10000.0)
    assert np.all(p["pos"][:, 2] == -1.0) and np.all(np.abs(p["pos"][:, :2]) <= 0.1)
    for a in range(2):
        assert stats.kstest(p["pos"][:, a], stats.uniform(-0.1, 0.2).cdf).pvalue > 1e-3
    assert np.all(p["dir"] == [0.0, 0.0, 1.0])


def test_field_calorimeter_mix():
    p = W.calo_field_primaries()
    counts = np.bincount(p["type"], minlength=3)
    assert stats.chisquare(counts).pvalue > 1e-3
    assert np.all((p["T"] >= 1000.0) & (p["T"] < 1e5))
    assert stats.kstest(np.log(p["T"] / 1000.0) / np.log(100.0), "uniform").pvalue > 1e-3
    assert _unit(p["dir"])
    theta = np.arccos(np.clip(p["dir"][:, 2], -1, 1))
    assert stats.kstest(theta / np.deg2rad(10.0), "uniform").pvalue > 1e-3
    phi = np.arctan2(p["dir"][:, 1], p["dir"][:, 0])
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3


def test_isotropic_point_source():
    p = W.cms_primaries()
    assert len(p["T"]) == 100 * 1000 and np.all(p["T"] == 1000.0) and np.all(p["type"] == W.GAMMA)
    assert np.array_equal(np.bincount(p["event"]), np.full(100, 1000))
    assert np.all(p["pos"] == 0.0) and _unit(p["dir"])
    assert stats.kstest((p["dir"][:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    phi = np.arctan2(p["dir"][:, 1], p["dir"][:, 0])
    assert stats.kstest((phi + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3
    # the mean direction vanishes (no preferred axis)
    assert np.all(np.abs(p["dir"].mean(0)) < 5 / np.sqrt(len(p["T"])))


def test_uneven_events_and_arrivals():
    p = W.batched_primaries()
    sizes = np.bincount(p["event"], minlength=256)
    assert sizes.min() >= 1 and sizes.max() <= 64 and len(sizes) == 256
    assert np.all(np.diff(p["event"]) >= 0)  # grouped by event
    assert np.all((p["T"] >= 100.0) & (p["T"] < 1e5))
    t = W.poisson_arrivals(100.0, 60.0)
    assert np.all(np.diff(t) > 0) and t[-1] < 60.0
    assert abs(len(t) - 6000) < 5 * np.sqrt(6000)
    assert stats.kstest(np.diff(t) * 100.0, "expon").pvalue > 1e-3


def test_subset_renumbers_events():
    """Listed events become 0, 1, ... in the listed order; each stays one
    contiguous run of primaries."""
    p = W.batched_primaries()
    sub = W.subset(p, [5, 2, 9])
    sizes = np.bincount(p["event"])
    assert np.array_equal(np.bincount(sub["event"]), sizes[[5, 2, 9]])
    runs = np.flatnonzero(np.diff(sub["event"])) + 1
    assert len(runs) == 2  # three contiguous runs
    assert np.array_equal(sub["T"][sub["event"] == 0], p["T"][p["event"] == 5])
