"""FP64 CPU oracle of the EM transport loop (arXiv:2203.09467, Secs. 2.1-3.2).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check, the
CPU-baseline leg of the benchmark and oracle/census.py (a count of the
step's FP64 operations) import this package.  It shares no code with the
GPU library and imports nothing from it.

Functions without a pin: absolute agreement of the closed-form physics with
measured data or Geant4 is "parity unpinned" (no data to check it is
available).  Every other function is pinned by tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emt_oracle.c")
_HDR = os.path.join(_HERE, "emt_oracle.h")
_LIB = os.path.join(_HERE, "libemt_oracle.so")
_lock = threading.Lock()
_lib = None

# process ids of orc_sample (7, 8: with the angular option)
PHOTO, COMPTON, PAIR, IONI, BREMS, ANNIH, BHABHA, BREMS_ANGULAR, PAIR_ANGULAR, RAYLEIGH, PHOTO_ANGULAR = range(11)
ALL_PROCESSES = 63
MSC = 64          # process-mask bit: multiple scattering of e+-
ANGULAR = 128     # process-mask bit: angular distributions of brems, pair, photoelectron
RAYLEIGH_BIT = 256  # process-mask bit: Rayleigh scattering


def _stale() -> bool:
    return (not os.path.exists(_LIB)) or any(os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math).
    Concurrent callers (processes of a multi-rank test) serialise on a lock
    file and write distinct temporaries."""
    if not (force or _stale()):
        return _LIB
    import fcntl
    with open(_LIB + ".lock", "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if force or _stale():
            tmp = f"{_LIB}.{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                   "-pthread", "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
            subprocess.check_call(cmd)
            os.replace(tmp, _LIB)
    return _LIB


def bind(L):
    """Declare the oracle's C functions on a loaded library (ctypes)."""
    d, u32, u64, i32, p = (ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p)
    sig = {
        "orc_philox4x32_10": (None, [p, p, p]),
        "orc_track_uniform": (d, [u32, u64, u64, u32, u32]),
        "orc_child_uid": (u64, [u32, u64, u64, u32, u32]),
        "orc_x0_gcm2": (d, [d, d]),
        "orc_sigma_kn": (d, [d]),
        "orc_dsigma_kn_deps": (d, [d, d]),
        "orc_sigma_pair_atom": (d, [d, d, d]),
        "orc_dsigma_pair_dx": (d, [d, d, d, d]),
        "orc_sigma_photo_atom": (d, [d, d, d]),
        "orc_sigma_moller": (d, [d, d]),
        "orc_dsigma_moller_deps": (d, [d, d]),
        "orc_sigma_bhabha": (d, [d, d]),
        "orc_dsigma_bhabha_deps": (d, [d, d]),
        "orc_sigma_heitler": (d, [d]),
        "orc_dsigma_heitler_deps": (d, [d, d]),
        "orc_sigma_brems_macro": (d, [d, d, d]),
        "orc_dsigma_brems_macro_dk": (d, [d, d, d]),
        "orc_dedx_rad": (d, [d, d, d]),
        "orc_dedx_coll": (d, [d, d, d, d, i32, d, d]),
        "orc_gauss_legendre": (None, [i32, p, p]),
        "orc_sample": (i32, [i32, d, d, d, u32, u64, u64, u32, p]),
        "orc_highland": (d, [d, d, d]),
        "orc_sigma_rayleigh_atom": (d, [d, d]),
        "orc_dsigma_rayleigh_dx": (d, [d, d, d]),
        "orc_msc": (i32, [d, d, d, u32, u64, u64, u32, p]),
        "orc_create": (p, [p, i32, p, p, i32, p, u32]),
        "orc_destroy": (None, [p]),
        "orc_grid_size": (i32, [p]),
        "orc_get_table": (i32, [p, i32, i32, i32, p]),
        "orc_range": (d, [p, i32, i32, d]),
        "orc_inv_range": (d, [p, i32, i32, d]),
        "orc_run": (i32, [p, i32, p, p, p, p, p, i32, p, p, p, i32, p, i32]),
        "orc_nav_exit": (i32, [p, i32, p, p, p]),
        "orc_locate": (i32, [p, p]),
        "orc_step_one": (i32, [p, p, u64, u64, p, p, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(ctypes.CDLL(_LIB))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- RNG
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def track_uniform(seed, event_id, uid, step, j) -> float:
    return lib().orc_track_uniform(seed, event_id, uid, step, j)


def child_uid(seed, event_id, uid, step, k) -> int:
    return lib().orc_child_uid(seed, event_id, uid, step, k)


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def sample(process: int, E: float, cut_e: float, cut_g: float, seed: int, event_id: int,
           uid: int, step: int = 0) -> np.ndarray:
    """One interaction from the draw stream of (event, uid, step).

    For PHOTO the `cut_e` argument is the binding energy.  Output layout:
    {E_after, dir[3], n, (type, T, dir[3]) x 2, local}."""
    out = np.zeros(16)
    lib().orc_sample(process, E, cut_e, cut_g, seed, event_id, uid, step, _ptr(out))
    return out


def highland(T, s, x0_cm) -> float:
    return lib().orc_highland(T, s, x0_cm)


def msc(T, s, x0_cm, direction, seed, event_id, uid, step=0) -> np.ndarray:
    """Direction after multiple scattering over a step of length s."""
    d = np.ascontiguousarray(direction, np.float64).copy()
    lib().orc_msc(T, s, x0_cm, seed, event_id, uid, step, _ptr(d))
    return d


# ---------------------------------------------------------------- setup
class Oracle:
    """Tables + geometry + transport.  Arguments are plain arrays:

    materials : (n, 5)  Z, A, rho, I_eV, bk_MeV   (rho == 0: vacuum)
    physics   : (9,)    cut_g, cut_em, cut_ep, e_lo, e_hi, bins_per_decade,
                        step_frac, final_range, process_mask
    layers    : (L, 3)  material, thickness_cm, score_bin
    world     : (21,)   z0, half_x, half_y, wlo[3], whi[3], B[3],
                        rk_delta_cm, max_steps, n_bins, max_field_step_cm,
                        geometry (0 layers, 1 cylinders), half_z_cm,
                        score_z, score_z_lo_cm, score_z_hi_cm
                        (a 16-entry world is layers scored per volume)
    """

    def __init__(self, materials, physics, layers, world, seed: int):
        self.materials = np.ascontiguousarray(materials, np.float64).reshape(-1, 5)
        self.physics = np.ascontiguousarray(physics, np.float64)
        self.layers = np.ascontiguousarray(layers, np.float64).reshape(-1, 3)
        w = np.zeros(21)
        w[: len(world)] = np.asarray(world, np.float64)
        self.world = w
        self.seed = int(seed)
        self.n_bins = int(self.world[14])
        h = lib().orc_create(_ptr(self.materials), len(self.materials), _ptr(self.physics),
                             _ptr(self.layers), len(self.layers), _ptr(self.world), self.seed)
        if not h:
            raise ValueError("orc_create rejected the configuration")
        self._h = h

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def grid_size(self) -> int:
        return lib().orc_grid_size(self._h)

    def table(self, m: int, p: int, q: int) -> np.ndarray:
        out = np.zeros(self.grid_size)
        if lib().orc_get_table(self._h, m, p, q, _ptr(out)) < 0:
            raise IndexError((m, p, q))
        return out

    def grid(self) -> np.ndarray:
        return self.table(0, 0, 5)

    def range(self, m, ci, T) -> float:
        return lib().orc_range(self._h, m, ci, T)

    def inv_range(self, m, ci, r) -> float:
        return lib().orc_inv_range(self._h, m, ci, r)

    def nav_exit(self, vol: int, p, d):
        """(t, next volume) of the exit from volume vol along d from p."""
        pp = np.ascontiguousarray(p, np.float64)
        dd = np.ascontiguousarray(d, np.float64)
        t = np.zeros(1)
        nxt = lib().orc_nav_exit(self._h, vol, _ptr(pp), _ptr(dd), _ptr(t))
        return float(t[0]), int(nxt)

    def locate(self, p) -> int:
        pp = np.ascontiguousarray(p, np.float64)
        return int(lib().orc_locate(self._h, _ptr(pp)))

    def run(self, prim: dict, n_events: int, event_ids, n_threads: int = 0, step_bins: int = 0):
        """Transport all events; returns (hist[n_events, n_bins], summary[n_events, 6]),
        plus the steps-per-track histogram [3, step_bins] when step_bins > 0."""
        ev = np.ascontiguousarray(prim["event"], np.int32)
        ty = np.ascontiguousarray(prim["type"], np.int32)
        T = np.ascontiguousarray(prim["T"], np.float64)
        pos = np.ascontiguousarray(prim["pos"], np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(prim["dir"], np.float64).reshape(-1, 3)
        ids = np.ascontiguousarray(event_ids, np.uint64)
        hist = np.zeros((n_events, self.n_bins))
        summ = np.zeros((n_events, 6))
        sh = np.zeros((3, max(step_bins, 1)), np.uint64)
        rc = lib().orc_run(self._h, len(ev), _ptr(ev), _ptr(ty), _ptr(T), _ptr(pos), _ptr(d),
                           n_events, _ptr(ids), _ptr(hist), _ptr(summ), n_threads,
                           _ptr(sh) if step_bins > 0 else None, step_bins)
        if rc != 0:
            raise ValueError("orc_run failed")
        if step_bins > 0:
            return hist, summ, sh
        return hist, summ

    def step_one(self, track, uid: int, event_id: int, with_uids: bool = False):
        """One step of one track; track = [type, T, x, y, z, ux, uy, uz, vol,
        step].  Returns (track after, secondaries, info[8] = {s, edep,
        boundary, interacted, process, alive, escaped, killed}[, sec uids])."""
        t = np.ascontiguousarray(track, np.float64).copy()
        sec = np.zeros(16)
        sec_uid = np.zeros(2, np.uint64)
        info = np.zeros(8)
        n = lib().orc_step_one(self._h, _ptr(t), uid, event_id, _ptr(sec), _ptr(sec_uid), _ptr(info))
        if with_uids:
            return t, sec[: 8 * n].reshape(n, 8), info, sec_uid[:n].copy()
        return t, sec[: 8 * n].reshape(n, 8), info
