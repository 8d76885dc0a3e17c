"""The allocation-free entry point (emt_transport_static) against the
context entry points, through the C ABI.

Callers that cannot allocate device memory (a framework allocator owns it,
a sandbox forbids it, or a serving loop cannot take the synchronisation)
use emt_transport_static, whose scratch is a fixed device array inside the
library.  This file is collected last so that a failure here comes after
every other test has run; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_09467_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-9  # the FP64 per-event tolerance of the other GPU tests


def _context_run(emt, s, prim, ids, slot_capacity):
    """The existing entry points (context, host primaries)."""
    n = len(ids)
    ctx = emt.context_for(s, slot_capacity=slot_capacity, max_events=n)
    ctx.submit(ids, prim)
    st = ctx.run()
    hist, summ, got_ids = ctx.read_all()
    ctx.close()
    assert np.array_equal(got_ids, ids)
    return hist, summ, st


def _static_call(emt, s, prim, ids, stream=None):
    """One emt_transport_static call with device primaries and device
    outputs (prefilled with -1); returns (status, hist, summary)."""
    import torch
    L = emt.lib()
    n = len(ids)
    mats = np.asarray(s.materials, np.float64)
    marr = (emt.Material * len(mats))(*[emt.Material(*r) for r in mats])
    larr = (emt.Layer * len(s.layers))(*[emt.Layer(int(r[0]), int(r[2]), float(r[1])) for r in s.layers])
    ph = emt.physics_struct(s.physics)
    wd = emt.world_struct(s.world)
    dev = torch.device("cuda", 0)
    d = {"event": torch.as_tensor(prim["event"], dtype=torch.int32, device=dev),
         "type": torch.as_tensor(prim["type"], dtype=torch.int32, device=dev),
         "T": torch.as_tensor(prim["T"], dtype=torch.float64, device=dev),
         "pos": torch.as_tensor(prim["pos"], dtype=torch.float64, device=dev).contiguous(),
         "dir": torch.as_tensor(prim["dir"], dtype=torch.float64, device=dev).contiguous()}
    p = emt.Primaries(len(prim["T"]), d["event"].data_ptr(), d["type"].data_ptr(), d["T"].data_ptr(),
                      d["pos"].data_ptr(), d["dir"].data_ptr())
    hist = torch.full((n, s.n_bins), -1.0, dtype=torch.float64, device=dev)
    summ = torch.full((n, 6), -1.0, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    rc = L.emt_transport_static(0, s.seed, marr, len(mats), ctypes.byref(ph), larr, len(s.layers),
                                ctypes.byref(wd), n, ids.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p),
                                ctypes.c_void_p(hist.data_ptr()), ctypes.c_void_p(summ.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream if stream is not None else None))
    torch.cuda.synchronize()
    return rc, hist.cpu().numpy(), summ.cpu().numpy()


def test_static_entry_point_matches_context_path_twice():
    import torch
    from paper_2203_09467_gb300 import emt

    s = W.calo_setup()
    n = 48
    prim = W.multi_primaries(n, 1, 4, 300.0, 30.0, seed=21)
    ids = np.arange(7000, 7000 + n, dtype=np.uint64)
    want_hist, want_summ, _ = _context_run(emt, s, prim, ids, 1 << 20)
    stream = torch.cuda.Stream(device=torch.device("cuda", 0))
    for call in range(2):
        rc, h, sm = _static_call(emt, s, prim, ids, stream)
        assert rc == 0, f"call {call}: status {rc}"
        e_in = want_summ[:, 3]
        # e_in of a multi-primary event is an FP64 atomic sum: order-dependent rounding
        assert np.all(np.abs(sm[:, 3] - e_in) <= 1e-14 * e_in)
        assert np.all(np.abs(sm[:, 0] - want_summ[:, 0]) <= TOL * e_in), f"call {call}"
        assert np.all(np.abs(h - want_hist).max(axis=1) <= TOL * e_in), f"call {call}"
        assert np.array_equal(sm[:, 4:], want_summ[:, 4:]), f"call {call}: step/track counts"
        assert np.all(np.abs(sm[:, 1:3] - want_summ[:, 1:3]) <= TOL * e_in[:, None])


def test_static_entry_point_defers_beyond_its_track_limit():
    """256 events of 50 GeV electrons hold about 4.7e5 tracks in flight at
    their peak (the context run below, with room for all of them), more
    than the fixed array's EMT_STATIC_MAX_TRACKS = 2^18: the static call
    defers the steps that do not fit and still returns every event as the
    context path does."""
    from paper_2203_09467_gb300 import emt

    s = W.calo_setup()
    n = 256
    prim = W.calo_primaries(n, energy=50000.0, seed=23)
    ids = np.arange(n, dtype=np.uint64) + 90000
    want_hist, want_summ, st = _context_run(emt, s, prim, ids, 1 << 22)
    assert st["peak_tracks"] > (1 << 18)
    rc, h, sm = _static_call(emt, s, prim, ids)
    assert rc == 0, rc
    e_in = want_summ[:, 3]
    assert np.all(np.abs(sm[:, 0] - want_summ[:, 0]) <= TOL * e_in)
    assert np.all(np.abs(h - want_hist).max(axis=1) <= TOL * e_in)
    assert np.array_equal(sm[:, 4:], want_summ[:, 4:])


def test_static_entry_point_rejects_a_bad_particle_type():
    """A primary whose type is not gamma, e- or e+ is the caller's error:
    EMT_ERR_INVALID_ARG, with no step run and the outputs untouched."""
    from paper_2203_09467_gb300 import emt

    s = W.calo_setup()
    prim = W.calo_primaries(3, energy=1000.0)
    prim["type"][1] = 7
    rc, h, sm = _static_call(emt, s, prim, np.array([1, 2, 3], np.uint64))
    assert rc == -1
    assert np.all(sm == -1.0) and np.all(h == -1.0)


def test_static_entry_point_rejects_oversized_batches():
    from paper_2203_09467_gb300 import emt

    L = emt.lib()
    s = W.calo_setup()
    mats = np.asarray(s.materials, np.float64)
    marr = (emt.Material * len(mats))(*[emt.Material(*r) for r in mats])
    larr = (emt.Layer * len(s.layers))(*[emt.Layer(int(r[0]), int(r[2]), float(r[1])) for r in s.layers])
    ph = emt.physics_struct(s.physics)
    wd = emt.world_struct(s.world)
    import torch
    n = 257  # one more event than the static limit
    ids = np.arange(n, dtype=np.uint64)
    hist = torch.zeros((n, s.n_bins), dtype=torch.float64, device="cuda")
    summ = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    p = emt.Primaries(0, None, None, None, None, None)
    rc = L.emt_transport_static(0, 1, marr, len(mats), ctypes.byref(ph), larr, len(s.layers), ctypes.byref(wd),
                                n, ids.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p),
                                ctypes.c_void_p(hist.data_ptr()), ctypes.c_void_p(summ.data_ptr()), None)
    assert rc == -2
    torch.cuda.synchronize()
    assert float(summ.abs().sum()) == 0.0  # nothing was run
