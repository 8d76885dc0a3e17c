"""FP64 operation census of the oracle's transport step.

MEASUREMENT INFRASTRUCTURE (like the oracle itself, it calls nothing but
oracle/): builds census.cpp (the oracle's own source with every double
counted) and transports a workload through it single-threaded, with the
same results as the oracle, bit for bit.  The counts per track-step are the
algorithmic FP64 work of the method, fixed by its definition and
independent of any GPU code; the step kernels' arithmetic roofline is
measured against them.

    python oracle/census.py [workload ...]     (calo, calo_field, cms, slab, batched)

prints one JSON line per workload: operations of each kind per track-step,
flops per track-step (add, sub, mul, div and sqrt one each, fma two) and the
elementary functions per track-step.
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

KINDS = ["add", "sub", "mul", "div", "fma", "sqrt", "cmp", "neg", "minmax", "round", "cbrt", "log", "exp", "log1p",
         "expm1", "sin", "cos", "pow"]
LIB = os.path.join(HERE, "libemt_oracle_census.so")


def build() -> str:
    src = os.path.join(HERE, "census.cpp")
    deps = [src, os.path.join(HERE, "emt_oracle.c"), os.path.join(HERE, "emt_oracle.h")]
    if not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in deps):
        tmp = f"{LIB}.{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c++17",
                               "-pthread", "-fpermissive", "-w", "-o", tmp, src, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def census(setup, prim, n_events):
    """Counts per track-step of one run of the workload, and the run's
    summary (which must equal the oracle's)."""
    L = oracle.bind(ctypes.CDLL(build()))
    L.orc_census_enable.argtypes = [ctypes.c_int]
    L.orc_census_read.argtypes = [ctypes.c_void_p, ctypes.c_int]
    saved = oracle._lib
    oracle._lib = L
    try:
        o = oracle.Oracle(setup.materials, setup.physics, setup.layers, setup.world, setup.seed)
        L.orc_census_reset()
        L.orc_census_enable(1)
        hist, summ = o.run(prim, n_events, np.arange(n_events), n_threads=1)
        L.orc_census_enable(0)
        counts = np.zeros(len(KINDS), np.uint64)
        L.orc_census_read(counts.ctypes.data_as(ctypes.c_void_p), len(KINDS))
        o.close()
    finally:
        oracle._lib = saved
    steps = float(summ[:, 4].sum())
    per = {k: float(c) / steps for k, c in zip(KINDS, counts)}
    flops = per["add"] + per["sub"] + per["mul"] + per["div"] + per["sqrt"] + 2.0 * per["fma"]
    elem = sum(per[k] for k in ("log", "exp", "log1p", "expm1", "sin", "cos", "pow"))
    return {"track_steps": steps, "per_track_step": per, "flops_per_track_step": flops,
            "fp64_ops_per_track_step": flops - per["fma"], "elementary_per_track_step": elem}, hist, summ


def main():
    from paper_2203_09467_gb300 import workloads as W
    names = sys.argv[1:] or ["calo", "calo_field", "cms"]
    for name in names:
        if name == "calo":
            s, n = W.calo_setup(), 200
            prim = W.calo_primaries(n)
        elif name == "calo_field":
            s, n = W.calo_field_setup(), 100
            prim = W.calo_field_primaries(n)
        elif name == "slab":
            s, n = W.slab_setup(), 1000
            prim = W.slab_primaries(n)
        elif name == "batched":
            # the first 6 of the 256 uneven events (1-64 primaries,
            # 0.1-100 GeV) of the batched calorimeter-in-2-T workload
            s, n = W.calo_field_setup(), 6
            s.seed = 4
            prim = W.subset(W.batched_primaries(256, seed=4), np.arange(n))
        else:
            s, n = W.cms_setup(), 4
            prim = W.cms_primaries(n, 1000)
        out, hist, summ = census(s, prim, n)
        # the census build computes exactly what the oracle computes
        ref = oracle.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
        rh, rs = ref.run(prim, n, np.arange(n), n_threads=1)
        out["identical_to_oracle"] = bool(np.array_equal(rs, summ) and np.array_equal(rh, hist))
        out["workload"] = name
        out["events"] = n
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
