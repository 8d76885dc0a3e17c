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


def test_static_entry_point_matches_context_path_twice():
    import torch
    from paper_2203_09467_gb300 import emt

    L = emt.lib()
    s = W.calo_setup()
    n = 48
    prim = W.multi_primaries(n, 1, 4, 300.0, 30.0, seed=21)
    ids = np.arange(7000, 7000 + n, dtype=np.uint64)

    # existing entry points (context, host primaries)
    ctx = emt.context_for(s, slot_capacity=1 << 20, max_events=n)
    ctx.submit(ids, prim)
    ctx.run()
    want_hist, want_summ, got_ids = ctx.read_all()
    ctx.close()
    assert np.array_equal(got_ids, ids)

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
    stream = torch.cuda.Stream(device=dev)
    for call in range(2):
        hist = torch.full((n, s.n_bins), -1.0, dtype=torch.float64, device=dev)
        summ = torch.full((n, 6), -1.0, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc = L.emt_transport_static(0, s.seed, marr, len(mats), ctypes.byref(ph), larr, len(s.layers),
                                    ctypes.byref(wd), n, ids.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p),
                                    ctypes.c_void_p(hist.data_ptr()), ctypes.c_void_p(summ.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, f"call {call}: status {rc}"
        torch.cuda.synchronize()
        h, sm = hist.cpu().numpy(), summ.cpu().numpy()
        e_in = want_summ[:, 3]
        # e_in of a multi-primary event is an FP64 atomic sum: order-dependent rounding
        assert np.all(np.abs(sm[:, 3] - e_in) <= 1e-14 * e_in)
        assert np.all(np.abs(sm[:, 0] - want_summ[:, 0]) <= TOL * e_in), f"call {call}"
        assert np.all(np.abs(h - want_hist).max(axis=1) <= TOL * e_in), f"call {call}"
        assert np.array_equal(sm[:, 4:], want_summ[:, 4:]), f"call {call}: step/track counts"
        assert np.all(np.abs(sm[:, 1:3] - want_summ[:, 1:3]) <= TOL * e_in[:, None])


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
