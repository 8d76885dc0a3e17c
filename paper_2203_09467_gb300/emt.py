"""Python binding of the C ABI in include/emt.h (argument marshalling only).

Every step of the transport runs in the CUDA library libemt.so; this module
converts arrays to the ABI's structs and pointers.  PyTorch provides the
device memory pool and the CUDA stream of a context.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HOST, DEVICE = 0, 1
PRECISION = {"fp64": 0, "mixed": 1}
LOOP = {"plain": 0, "graph": 1, "persistent": 2}
SCHEDULE = {"fused": 0, "split": 1, "pipelined": 2}
SELECT = {"order": 0, "low_energy": 1}
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "CAPACITY", -3: "CUDA", -4: "BAD_STATE", -5: "TIMEOUT",
          -6: "NOT_READY", -7: "HOST_OOM"}
SUMMARY_FIELDS = ("edep", "escaped", "killed", "e_in", "n_steps", "n_tracks")


class EmtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("precision", ctypes.c_int32), ("slot_capacity", ctypes.c_int64),
                ("max_events", ctypes.c_int32), ("max_bins", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("loop_mode", ctypes.c_int32), ("graph_steps", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("seed", ctypes.c_uint32),
                ("cuda_stream", ctypes.c_void_p), ("device_pool", ctypes.c_void_p), ("pool_bytes", ctypes.c_size_t),
                ("step_hist_bins", ctypes.c_int32), ("select_policy", ctypes.c_int32),
                ("max_active", ctypes.c_int64), ("spill_above", ctypes.c_int64)]


class Material(ctypes.Structure):
    _fields_ = [("Z", ctypes.c_double), ("A_g_mol", ctypes.c_double), ("rho_g_cm3", ctypes.c_double),
                ("I_eV", ctypes.c_double), ("bk_MeV", ctypes.c_double)]


class Physics(ctypes.Structure):
    _fields_ = [("cut_MeV", ctypes.c_double * 3), ("grid_lo_MeV", ctypes.c_double), ("grid_hi_MeV", ctypes.c_double),
                ("bins_per_decade", ctypes.c_int32), ("process_mask", ctypes.c_uint32), ("step_frac", ctypes.c_double),
                ("final_range_cm", ctypes.c_double)]


class Layer(ctypes.Structure):
    _fields_ = [("material", ctypes.c_int32), ("score_bin", ctypes.c_int32), ("thickness_cm", ctypes.c_double)]


class World(ctypes.Structure):
    _fields_ = [("z0_cm", ctypes.c_double), ("half_x_cm", ctypes.c_double), ("half_y_cm", ctypes.c_double),
                ("lo_cm", ctypes.c_double * 3), ("hi_cm", ctypes.c_double * 3), ("B_tesla", ctypes.c_double * 3),
                ("rk_delta_cm", ctypes.c_double), ("max_field_step_cm", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("n_bins", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("score_z", ctypes.c_int32), ("half_z_cm", ctypes.c_double), ("score_z_lo_cm", ctypes.c_double),
                ("score_z_hi_cm", ctypes.c_double)]


class Primaries(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("event", ctypes.c_void_p), ("type", ctypes.c_void_p),
                ("T_MeV", ctypes.c_void_p), ("pos_cm", ctypes.c_void_p), ("dir", ctypes.c_void_p)]


class ServeOptions(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("steps_per_poll", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("time_scale", ctypes.c_double), ("admit_below", ctypes.c_int64)]


SERVE = {"continuous": 0, "batch": 1}


class StepRecord(ctypes.Structure):
    _fields_ = [("photons", ctypes.c_int64), ("charged", ctypes.c_int64), ("interacting", ctypes.c_int64),
                ("deferred", ctypes.c_int64), ("held", ctypes.c_int64), ("ms", ctypes.c_double)]


class RunStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("track_steps", ctypes.c_int64), ("peak_tracks", ctypes.c_int64),
                ("deferred", ctypes.c_int64), ("live_tracks", ctypes.c_int64), ("state_bytes", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int32), ("held", ctypes.c_int64),
                ("spilled", ctypes.c_int64), ("peak_spilled", ctypes.c_int64), ("rk4_substeps", ctypes.c_int64)]


_lib = None

# every symbol the header declares, with its ctypes signature
_SIGS = {
    "emt_default_options": (None, [ctypes.POINTER(Options)]),
    "emt_pool_bytes": (ctypes.c_size_t, [ctypes.POINTER(Options)]),
    "emt_create": (ctypes.c_int32, [ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)]),
    "emt_destroy": (None, [ctypes.c_void_p]),
    "emt_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "emt_load_materials": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(Material), ctypes.c_int32,
                                            ctypes.POINTER(Physics)]),
    "emt_load_geometry": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(Layer), ctypes.c_int32,
                                           ctypes.POINTER(World)]),
    "emt_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(Primaries),
                                    ctypes.c_int32]),
    "emt_run": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(RunStats)]),
    "emt_run_traced": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(RunStats),
                                        ctypes.POINTER(StepRecord), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "emt_read_step_hist": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "emt_poll": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "emt_read_event": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "emt_read_all": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int32]),
    "emt_events_in_flight": (ctypes.c_int32, [ctypes.c_void_p]),
    "emt_tracks_in_flight": (ctypes.c_int64, [ctypes.c_void_p]),
    "emt_get_table": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "emt_debug_set_tracks": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "emt_debug_get_tracks": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "emt_serve": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Primaries),
                                   ctypes.POINTER(ServeOptions), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "emt_debug_wait_timeout": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    "emt_measure_dfma_rate": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_double)]),
    "emt_measure_fp64_op_rates": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.POINTER(ctypes.c_double)]),
    "emt_transport_static": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(Material),
                                              ctypes.c_int32, ctypes.POINTER(Physics), ctypes.POINTER(Layer),
                                              ctypes.c_int32, ctypes.POINTER(World), ctypes.c_int32,
                                              ctypes.c_void_p, ctypes.POINTER(Primaries), ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libemt.so (building it in-tree if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library {_build.LIB} is missing; run paper_2203_09467_gb300.build")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """Pointer of a contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(ctypes.c_void_p)
    assert a.is_contiguous()
    return ctypes.c_void_p(a.data_ptr())


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def physics_struct(physics) -> Physics:
    ph = np.asarray(physics, np.float64)
    s = Physics()
    for k in range(3):
        s.cut_MeV[k] = ph[k]
    s.grid_lo_MeV, s.grid_hi_MeV = ph[3], ph[4]
    s.bins_per_decade = int(ph[5])
    s.step_frac, s.final_range_cm = ph[6], ph[7]
    s.process_mask = int(ph[8])
    return s


def world_struct(world) -> World:
    w = np.asarray(world, np.float64)
    s = World()
    s.z0_cm, s.half_x_cm, s.half_y_cm = w[0], w[1], w[2]
    for a in range(3):
        s.lo_cm[a], s.hi_cm[a], s.B_tesla[a] = w[3 + a], w[6 + a], w[9 + a]
    s.rk_delta_cm = w[12]
    s.max_steps = int(w[13])
    s.n_bins = int(w[14])
    s.max_field_step_cm = w[15]
    if len(w) >= 21:
        s.geometry = int(w[16])
        s.half_z_cm = w[17]
        s.score_z = int(w[18])
        s.score_z_lo_cm, s.score_z_hi_cm = w[19], w[20]
    return s


class Context:
    """One transport context on one GPU (emt_create ... emt_destroy)."""

    def __init__(self, *, device: int = 0, precision: str = "fp64", slot_capacity: int = 1 << 22,
                 max_events: int = 10000, max_bins: int = 128, block_size: int = 0, loop_mode: str = "plain",
                 graph_steps: int = 12, seed: int = 1, use_torch_pool: bool = True, schedule: str = "fused",
                 step_hist_bins: int = 0, max_active: int = 0, select: str = "order", spill_above: int = 0):
        import torch
        L = lib()
        self._torch = torch
        o = Options()
        L.emt_default_options(ctypes.byref(o))
        o.device = device
        o.precision = PRECISION[precision]
        o.slot_capacity = int(slot_capacity)
        o.max_events = int(max_events)
        o.max_bins = int(max_bins)
        o.block_size = int(block_size)
        o.loop_mode = LOOP[loop_mode]
        o.graph_steps = int(graph_steps)
        o.schedule = SCHEDULE[schedule]
        o.seed = int(seed) & 0xFFFFFFFF
        o.step_hist_bins = int(step_hist_bins)
        o.max_active = int(max_active)
        o.select_policy = SELECT[select]
        o.spill_above = int(spill_above)
        self.device = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=self.device)
        o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.pool = None
        if use_torch_pool:
            nbytes = L.emt_pool_bytes(ctypes.byref(o))
            if nbytes == 0:
                raise EmtError(-1, "invalid options")
            self.pool = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.pool.data_ptr()
            o.device_pool = ctypes.c_void_p((base + 255) // 256 * 256)
            o.pool_bytes = nbytes
        self.options = o
        h = ctypes.c_void_p()
        rc = L.emt_create(ctypes.byref(o), ctypes.byref(h))
        if rc != 0:
            raise EmtError(rc, "emt_create failed")
        self._h = h
        self.n_bins = None
        self.precision = precision

    # -- helpers
    def _check(self, rc):
        if rc != 0:
            msg = lib().emt_last_error(self._h)
            raise EmtError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            lib().emt_destroy(self._h)
            self._h = None
            self.pool = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- set-up
    def load_materials(self, materials, physics):
        m = np.asarray(materials, np.float64).reshape(-1, 5)
        arr = (Material * len(m))(*[Material(*row) for row in m])
        ph = physics_struct(physics)
        self._check(lib().emt_load_materials(self._h, arr, len(m), ctypes.byref(ph)))

    def load_geometry(self, layers, world):
        ly = np.asarray(layers, np.float64).reshape(-1, 3)
        arr = (Layer * len(ly))(*[Layer(int(r[0]), int(r[2]), float(r[1])) for r in ly])
        w = world_struct(world)
        self._check(lib().emt_load_geometry(self._h, arr, len(ly), ctypes.byref(w)))
        self.n_bins = int(w.n_bins)

    def load(self, setup):
        """Materials, physics and geometry of a workloads.Setup."""
        self.load_materials(setup.materials, setup.physics)
        self.load_geometry(setup.layers, setup.world)

    # -- events
    def submit(self, event_ids, prim):
        """prim: dict of event/type/T/pos/dir as numpy (host) or CUDA tensors."""
        ids = np.ascontiguousarray(event_ids, np.uint64)
        if _is_torch_cuda(prim["T"]):
            where = DEVICE
            t = self._torch
            keep = {"event": prim["event"].to(t.int32).contiguous(), "type": prim["type"].to(t.int32).contiguous(),
                    "T": prim["T"].to(t.float64).contiguous(), "pos": prim["pos"].to(t.float64).contiguous(),
                    "dir": prim["dir"].to(t.float64).contiguous()}
            # the library reads device inputs on its own stream
            self.stream.wait_stream(t.cuda.current_stream(self.device))
        elif hasattr(prim["T"], "numpy"):
            where = HOST
            keep = {k: v.contiguous() for k, v in prim.items()}
        else:
            where = HOST
            keep = {"event": np.ascontiguousarray(prim["event"], np.int32),
                    "type": np.ascontiguousarray(prim["type"], np.int32),
                    "T": np.ascontiguousarray(prim["T"], np.float64),
                    "pos": np.ascontiguousarray(prim["pos"], np.float64),
                    "dir": np.ascontiguousarray(prim["dir"], np.float64)}
        p = Primaries(int(len(keep["T"])), _ptr(keep["event"]), _ptr(keep["type"]), _ptr(keep["T"]),
                      _ptr(keep["pos"]), _ptr(keep["dir"]))
        self._check(lib().emt_submit(self._h, len(ids), _ptr(ids), ctypes.byref(p), where))

    def run(self, max_iterations: int = 0) -> dict:
        st = RunStats()
        self._check(lib().emt_run(self._h, int(max_iterations), ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in RunStats._fields_}

    def run_traced(self, max_iterations: int = 0, cap: int = 1 << 16):
        """emt_run_traced: (stats, records[n, 6] = photons, charged,
        interacting, deferred, held, ms per iteration)."""
        st = RunStats()
        rec = (StepRecord * cap)()
        n = ctypes.c_int32()
        self._check(lib().emt_run_traced(self._h, int(max_iterations), ctypes.byref(st), rec, cap, ctypes.byref(n)))
        out = np.array([[r.photons, r.charged, r.interacting, r.deferred, r.held, r.ms] for r in rec[: n.value]],
                       np.float64).reshape(-1, 6)
        return {f: getattr(st, f) for f, _ in RunStats._fields_}, out

    def read_step_hist(self, reset: bool = False) -> np.ndarray:
        """Steps-per-track histogram [3, step_hist_bins] (gamma, e-, e+)."""
        nb = int(self.options.step_hist_bins)
        out = np.zeros((3, max(nb, 1)), np.uint64)
        self._check(lib().emt_read_step_hist(self._h, _ptr(out), nb, int(bool(reset))))
        return out

    def poll(self, cap: int = 65536):
        out = np.zeros(cap, np.uint64)
        n = ctypes.c_int32()
        self._check(lib().emt_poll(self._h, _ptr(out), cap, ctypes.byref(n)))
        return out[: n.value].copy()

    def read_event(self, event_id: int):
        hist = np.zeros(self.n_bins)
        summ = np.zeros(6)
        self._check(lib().emt_read_event(self._h, int(event_id), _ptr(hist), _ptr(summ)))
        return hist, summ

    def events_in_flight(self) -> int:
        return lib().emt_events_in_flight(self._h)

    def read_all(self, hist=None, summary=None):
        """Read every event in submission order.  With CUDA tensors hist
        (n, n_bins) and summary (n, 6) the results stay on the device."""
        n = self.events_in_flight()
        ids = np.zeros(max(n, 1), np.uint64)
        if hist is not None and _is_torch_cuda(hist):
            self._check(lib().emt_read_all(self._h, _ptr(hist), _ptr(summary), _ptr(ids), DEVICE))
            return hist, summary, ids[:n]
        if hist is None:
            hist = np.zeros((n, self.n_bins))
            summary = np.zeros((n, 6))
        self._check(lib().emt_read_all(self._h, _ptr(hist), _ptr(summary), _ptr(ids), HOST))
        return hist, summary, ids[:n]

    def serve(self, event_ids, arrival_s, prim, mode: str = "continuous", steps_per_poll: int = 8,
              time_scale: float = 1.0, admit_below: int = -1):
        """Replay a request stream (emt_serve).  prim: host primaries grouped
        by event in arrival order.  Returns admit_s, done_s, hist, summary."""
        ids = np.ascontiguousarray(event_ids, np.uint64)
        arr = np.ascontiguousarray(arrival_s, np.float64)
        n = len(ids)
        ev = np.asarray(prim["event"])
        count = np.bincount(ev, minlength=n).astype(np.int32)
        first = np.concatenate([[0], np.cumsum(count)[:-1]]).astype(np.int32)
        keep = {"type": np.ascontiguousarray(prim["type"], np.int32), "T": np.ascontiguousarray(prim["T"], np.float64),
                "pos": np.ascontiguousarray(prim["pos"], np.float64), "dir": np.ascontiguousarray(prim["dir"], np.float64),
                "event": np.ascontiguousarray(ev, np.int32)}
        p = Primaries(len(keep["T"]), _ptr(keep["event"]), _ptr(keep["type"]), _ptr(keep["T"]), _ptr(keep["pos"]),
                      _ptr(keep["dir"]))
        if admit_below < 0:  # default: a quarter of the track store
            admit_below = int(self.options.slot_capacity) // 4
        o = ServeOptions(SERVE[mode], int(steps_per_poll), int(self.n_bins), float(time_scale), int(admit_below))
        admit = np.zeros(n)
        done = np.zeros(n)
        hist = np.zeros((n, self.n_bins))
        summ = np.zeros((n, 6))
        self._check(lib().emt_serve(self._h, n, _ptr(ids), _ptr(arr), _ptr(first), _ptr(count), ctypes.byref(p),
                                    ctypes.byref(o), _ptr(admit), _ptr(done), _ptr(hist), _ptr(summ)))
        return admit, done, hist, summ

    # -- diagnostics
    def get_table(self, m: int, p: int, q: int) -> np.ndarray:
        out = np.zeros(256)
        n = ctypes.c_int32()
        self._check(lib().emt_get_table(self._h, m, p, q, _ptr(out), 256, ctypes.byref(n)))
        return out[: n.value].copy()

    def debug_set_tracks(self, rec, uid, event_slot):
        rec = np.ascontiguousarray(rec, np.float64).reshape(-1, 10)
        uid = np.ascontiguousarray(uid, np.uint64)
        sl = np.ascontiguousarray(event_slot, np.int32)
        self._check(lib().emt_debug_set_tracks(self._h, len(rec), _ptr(rec), _ptr(uid), _ptr(sl)))

    def debug_get_tracks(self, cap: int = 1 << 20):
        rec = np.zeros((cap, 10))
        uid = np.zeros(cap, np.uint64)
        sl = np.zeros(cap, np.int32)
        n = ctypes.c_int32()
        self._check(lib().emt_debug_get_tracks(self._h, cap, _ptr(rec), _ptr(uid), _ptr(sl), ctypes.byref(n)))
        k = n.value
        return rec[:k].copy(), uid[:k].copy(), sl[:k].copy()


def measure_dfma_rate(device: int = 0, iters: int = 4000, repeats: int = 5) -> float:
    """FP64 fused multiply-adds per second of the device (emt_measure_dfma_rate)."""
    out = ctypes.c_double()
    rc = lib().emt_measure_dfma_rate(int(device), int(iters), int(repeats), ctypes.byref(out))
    if rc != 0:
        raise EmtError(rc, "emt_measure_dfma_rate failed")
    return out.value


def context_for(setup, **kw) -> Context:
    """Context with the materials and geometry of a workloads.Setup loaded."""
    kw.setdefault("seed", setup.seed)
    kw.setdefault("max_bins", max(1, setup.n_bins))
    ctx = Context(**kw)
    ctx.load(setup)
    return ctx


def measure_fp64_op_rates(device: int = 0, iters: int = 256, repeats: int = 3) -> dict:
    """FP64 divisions and logarithms per second of the device, native and on
    the integer pipe (emt_measure_fp64_op_rates)."""
    out = (ctypes.c_double * 4)()
    rc = lib().emt_measure_fp64_op_rates(int(device), int(iters), int(repeats), out)
    if rc != 0:
        raise EmtError(rc, "emt_measure_fp64_op_rates failed")
    return {"div_native": out[0], "div_integer": out[1], "log_native": out[2], "log_integer": out[3]}
