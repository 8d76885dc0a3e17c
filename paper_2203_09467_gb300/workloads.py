"""Seeded synthetic workloads: materials, geometry and primaries.

This module holds input data only (material constants, layer stacks and the
random primaries of each workload); it contains none of the transport
arithmetic, and both the GPU library and the CPU oracle are fed from it.

Workloads (synthetic calorimeter workloads, plus the paper's own test
problem of Sec. 3.2 with its unstated dimensions read as below):

  slab      1,000 events x one 100 MeV e- along +z into a 5 cm Pb slab,
            20x20 cm, no field, one score bin.
  calo      10,000 events x one 10 GeV e- at normal incidence, x,y uniform
            within +-1 mm, 50 x (2 mm Pb + 5 mm LAr), 40x40 cm, 100 bins.
  calo_field  the calo stack in a uniform 2 T field along x; primaries
            e-/e+/gamma with equal probability, energy log-uniform
            1-100 GeV, polar angle uniform in [0, 10 deg], azimuth uniform.
  batched   256 events of 1-64 primaries, e-/e+/gamma, 0.1-100 GeV
            log-uniform, on the calo_field geometry.
  served    Poisson arrivals; 1-100 primaries per event, 1-50 GeV.
  cms       the paper's verification problem (Sec. 3.2): six concentric
            cylindrical shells about the z axis out to 375 cm, each one
            element (vacuum, Si, Pb, C, Ti, Fe), no field; 100 events x 1000
            photons of 1 GeV from an isotropic point source at the origin;
            energy deposition tallied along z.  The paper gives only the
            outer radius: the shell radii (30, 125, 175, 275, 325, 375 cm)
            and the half-length (700 cm) are readings of a CMS-like layout.
  cms_field the cms geometry in a uniform 3.8 T field along z.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Z, A (g/mol), rho (g/cm3), I (eV), K-shell binding (MeV).  Z, rho of Pb and
# LAr as given for the workloads; A, I and the K binding energies are the
# PDG / X-ray data booklet values.
VACUUM = (0.0, 1.0, 0.0, 1.0, 0.0)
LEAD = (82.0, 207.2, 11.35, 823.0, 0.0880)
LIQUID_ARGON = (18.0, 39.948, 1.396, 188.0, 0.0032)
SILICON = (14.0, 28.0855, 2.329, 173.0, 0.001839)
CARBON = (6.0, 12.0107, 2.21, 78.0, 0.000284)     # graphite
TITANIUM = (22.0, 47.867, 4.54, 233.0, 0.004966)
IRON = (26.0, 55.845, 7.874, 286.0, 0.007112)

GAMMA, ELECTRON, POSITRON = 0, 1, 2


@dataclasses.dataclass
class Setup:
    """Plain description of one workload's detector and physics options."""
    name: str
    materials: np.ndarray      # (n, 5)
    physics: np.ndarray        # (9,)  cut_g, cut_em, cut_ep, e_lo, e_hi, bpd, step_frac, final_range, mask
    layers: np.ndarray         # (L, 3) material, thickness_cm, score_bin
    world: np.ndarray          # (21,) z0, half_x, half_y, wlo[3], whi[3], B[3], rk_delta, max_steps, n_bins,
    #                            max_field_step, geometry, half_z, score_z, score_z_lo, score_z_hi
    seed: int

    @property
    def n_bins(self) -> int:
        return int(self.world[14])


def physics(cut=1.0, mask=63, e_lo=1e-3, e_hi=1e5, bpd=8, step_frac=0.2, final_range=0.1):
    return np.array([cut, cut, cut, e_lo, e_hi, bpd, step_frac, final_range, mask], np.float64)


GEOM_LAYERS, GEOM_CYLINDERS = 0, 1


def world(z0, half_x, half_y, wlo, whi, B=(0.0, 0.0, 0.0), rk_delta=1e-5, max_steps=100000,
          n_bins=100, max_field_step=10.0, geometry=GEOM_LAYERS, half_z=0.0, score_z=None):
    """score_z: None scores per volume; (lo, hi) scores n_bins equal bins of z."""
    zs = (0, 0.0, 0.0) if score_z is None else (1, float(score_z[0]), float(score_z[1]))
    return np.array([z0, half_x, half_y, *wlo, *whi, *B, rk_delta, max_steps, n_bins, max_field_step,
                     geometry, half_z, *zs], np.float64)


def slab_setup(seed=1, mask=63, cut=1.0, thickness=5.0) -> Setup:
    mats = np.array([LEAD], np.float64)
    layers = np.array([[0, thickness, 0]], np.float64)
    w = world(0.0, 10.0, 10.0, (-100.0, -100.0, -50.0), (100.0, 100.0, thickness + 50.0), n_bins=1)
    return Setup("slab", mats, physics(cut=cut, mask=mask), layers, w, seed)


def calo_layers(n_pairs=50, pb=0.2, lar=0.5):
    rows = []
    for i in range(n_pairs):
        rows.append([0, pb, 2 * i])
        rows.append([1, lar, 2 * i + 1])
    return np.array(rows, np.float64)


def calo_setup(seed=2, mask=63, n_pairs=50) -> Setup:
    mats = np.array([LEAD, LIQUID_ARGON], np.float64)
    layers = calo_layers(n_pairs)
    depth = float(layers[:, 1].sum())
    w = world(0.0, 20.0, 20.0, (-100.0, -100.0, -50.0), (100.0, 100.0, depth + 50.0), n_bins=100)
    return Setup("calo", mats, physics(mask=mask), layers, w, seed)


def calo_field_setup(seed=3, mask=63, n_pairs=50, B=2.0) -> Setup:
    mats = np.array([LEAD, LIQUID_ARGON], np.float64)
    layers = calo_layers(n_pairs)
    depth = float(layers[:, 1].sum())
    w = world(0.0, 20.0, 20.0, (-25.0, -25.0, -5.0), (25.0, 25.0, depth + 5.0), B=(B, 0.0, 0.0),
              n_bins=100, max_field_step=10.0)
    return Setup("calo_field", mats, physics(mask=mask), layers, w, seed)


CMS_RADII = (30.0, 125.0, 175.0, 275.0, 325.0, 375.0)
CMS_HALF_Z = 700.0


def cms_setup(seed=6, mask=63, B=0.0, n_bins=140) -> Setup:
    """Six single-element shells (vacuum, Si, Pb, C, Ti, Fe); layers are
    radial shells (thickness = radial extent), scored along z over the
    full length in n_bins bins."""
    mats = np.array([VACUUM, SILICON, LEAD, CARBON, TITANIUM, IRON], np.float64)
    r = (0.0,) + CMS_RADII
    layers = np.array([[i, r[i + 1] - r[i], i] for i in range(6)], np.float64)
    w = world(0.0, 0.0, 0.0, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), B=(0.0, 0.0, B), n_bins=n_bins,
              max_field_step=10.0, geometry=GEOM_CYLINDERS, half_z=CMS_HALF_Z,
              score_z=(-CMS_HALF_Z, CMS_HALF_Z))
    return Setup("cms" if B == 0.0 else "cms_field", mats, physics(mask=mask), layers, w, seed)


def cms_field_setup(seed=7, mask=63, B=3.8) -> Setup:
    return cms_setup(seed=seed, mask=mask, B=B)


# ---------------------------------------------------------------- primaries
def _empty():
    return {"event": [], "type": [], "T": [], "pos": [], "dir": []}


def _finish(p):
    return {
        "event": np.asarray(p["event"], np.int32),
        "type": np.asarray(p["type"], np.int32),
        "T": np.asarray(p["T"], np.float64),
        "pos": np.asarray(p["pos"], np.float64).reshape(-1, 3),
        "dir": np.asarray(p["dir"], np.float64).reshape(-1, 3),
    }


def _cone_dirs(rng, n, max_deg):
    theta = np.deg2rad(max_deg) * rng.random(n)
    phi = 2.0 * np.pi * rng.random(n)
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)


def slab_primaries(n_events=1000, energy=100.0, seed=1):
    del seed  # fully deterministic: every event is the same primary
    n = n_events
    return _finish({
        "event": np.arange(n), "type": np.full(n, ELECTRON), "T": np.full(n, energy),
        "pos": np.tile([0.0, 0.0, -1.0], (n, 1)), "dir": np.tile([0.0, 0.0, 1.0], (n, 1))})


def calo_primaries(n_events=10000, energy=10000.0, seed=2):
    rng = np.random.default_rng(seed)
    n = n_events
    xy = (2.0 * rng.random((n, 2)) - 1.0) * 0.1
    pos = np.concatenate([xy, np.full((n, 1), -1.0)], axis=1)
    return _finish({
        "event": np.arange(n), "type": np.full(n, ELECTRON), "T": np.full(n, energy),
        "pos": pos, "dir": np.tile([0.0, 0.0, 1.0], (n, 1))})


def calo_field_primaries(n_events=10000, seed=3, e_min=1000.0, e_ratio=100.0):
    rng = np.random.default_rng(seed)
    n = n_events
    types = rng.integers(0, 3, n)
    T = e_min * e_ratio ** rng.random(n)
    xy = (2.0 * rng.random((n, 2)) - 1.0) * 0.1
    pos = np.concatenate([xy, np.full((n, 1), -1.0)], axis=1)
    return _finish({"event": np.arange(n), "type": types, "T": T, "pos": pos,
                    "dir": _cone_dirs(rng, n, 10.0)})


def isotropic_dirs(rng, n):
    """Directions uniform on the unit sphere."""
    cost = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * np.pi * rng.random(n)
    sint = np.sqrt(np.maximum(0.0, 1.0 - cost * cost))
    return np.stack([sint * np.cos(phi), sint * np.sin(phi), cost], axis=1)


def cms_primaries(n_events=100, per_event=1000, energy=1000.0, seed=6, particle=GAMMA):
    """Isotropic point source at the origin: per_event photons of `energy`
    per event."""
    rng = np.random.default_rng(seed)
    n = n_events * per_event
    return _finish({
        "event": np.repeat(np.arange(n_events), per_event), "type": np.full(n, particle),
        "T": np.full(n, energy), "pos": np.zeros((n, 3)), "dir": isotropic_dirs(rng, n)})


def multi_primaries(n_events, n_min, n_max, e_min, e_ratio, seed, max_deg=10.0):
    """Events of uneven size: n_prim uniform in [n_min, n_max] per event."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(n_min, n_max + 1, n_events)
    n = int(counts.sum())
    ev = np.repeat(np.arange(n_events), counts)
    types = rng.integers(0, 3, n)
    T = e_min * e_ratio ** rng.random(n)
    xy = (2.0 * rng.random((n, 2)) - 1.0) * 0.1
    pos = np.concatenate([xy, np.full((n, 1), -1.0)], axis=1)
    return _finish({"event": ev, "type": types, "T": T, "pos": pos, "dir": _cone_dirs(rng, n, max_deg)})


def batched_primaries(n_events=256, seed=4):
    return multi_primaries(n_events, 1, 64, 100.0, 1000.0, seed)


def served_primaries(n_events, seed=5):
    return multi_primaries(n_events, 1, 100, 1000.0, 50.0, seed)


def poisson_arrivals(rate_hz, duration_s, seed=5):
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed + 1000)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        out.append(t)
    return np.asarray(out)


def subset(prim, events):
    """Primaries of the listed events, renumbered 0..len(events)-1."""
    events = np.asarray(events)
    remap = -np.ones(int(prim["event"].max()) + 1 if len(prim["event"]) else 0, np.int64)
    remap[events] = np.arange(len(events))
    keep = np.isin(prim["event"], events)
    out = {k: v[keep] for k, v in prim.items()}
    out["event"] = remap[out["event"]].astype(np.int32)
    order = np.argsort(out["event"], kind="stable")
    return {k: v[order] for k, v in out.items()}
