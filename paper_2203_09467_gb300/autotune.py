"""Autotuner of the step-loop launch configuration.

The tunable knobs are the step schedule (fused: one kernel regrouping the
interactions inside each block; split: a transport kernel and an
interaction kernel joined by a queue in device memory; pipelined: one
kernel per step that samples the previous step's queue while it transports
the current tracks), the block size (128
or 256 threads: a larger block regroups more interacting tracks per model, a
smaller one leaves more blocks per SM) and the step-loop driver (a host loop
with one counter read per step, CUDA graphs of 12 or 24 steps with one
counter read per graph, or the persistent kernel that runs up to 64 or 256
fused steps per launch with a grid barrier between steps).  Two more
candidates select the lowest-energy tracks (split schedule, at most 3/4 or
5/8 of the track store stepped per iteration): where the showers outgrow
the store, holding the most energetic tracks back lets the others finish
instead of deferring steps for want of a slot.  Every candidate
transports the same batch of events; the fastest by CUDA-event time wins.
Results are cached per GPU name, workload name, precision and track-store
size in a JSON file next to this module.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import emt

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")

CANDIDATES = [
    {"block_size": b, "loop_mode": loop, "graph_steps": k, "schedule": sched}
    for sched in ("fused", "split", "pipelined")
    for b in (128, 256)
    for loop, k in (("plain", 12), ("graph", 12), ("graph", 24))
] + [
    {"block_size": b, "loop_mode": "persistent", "graph_steps": k, "schedule": "fused"}
    for b in (128, 256)
    for k in (64, 256)
]


def selection_candidates(slot_capacity):
    """Low-energy track selection with budgets of 3/4 and 5/8 of the store
    (the second moves held tracks to host memory above 13/16)."""
    q = int(slot_capacity)
    return [
        {"block_size": 256, "loop_mode": "graph", "graph_steps": 24, "schedule": "split",
         "max_active": 3 * q // 4, "select": "low_energy"},
        {"block_size": 256, "loop_mode": "graph", "graph_steps": 24, "schedule": "split",
         "max_active": 5 * q // 8, "select": "low_energy", "spill_above": 13 * q // 16},
    ]


def _key(name, precision, slot_capacity):
    import torch
    return f"{torch.cuda.get_device_name()}|{name}|{precision}|{int(slot_capacity)}"


def time_config(setup, prim, ids, precision, cfg, repeats=2, slot_capacity=1 << 25, device=0):
    """Best-of-`repeats` milliseconds of one full transport of the batch."""
    import torch
    ctx = emt.context_for(setup, device=device, precision=precision, slot_capacity=slot_capacity,
                          max_events=len(ids), **cfg)
    dprim = {k: torch.as_tensor(v).to(ctx.device) for k, v in prim.items()}
    hist = torch.empty((len(ids), setup.n_bins), dtype=torch.float64, device=ctx.device)
    summ = torch.empty((len(ids), 6), dtype=torch.float64, device=ctx.device)
    best = float("inf")
    for _ in range(repeats + 1):  # the first pass warms up (and captures the graph)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(ctx.stream)
        ctx.submit(ids, dprim)
        ctx.run()
        ctx.read_all(hist, summ)
        b.record(ctx.stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    ctx.close()
    return best


def autotune(name, setup, prim, ids, precision="fp64", use_cache=True, repeats=2, slot_capacity=1 << 25,
             device=0, candidates=None):
    """Return (best configuration, {candidate: ms}) for this workload."""
    key = _key(name, precision, slot_capacity)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except Exception:
            cache = {}
    if use_cache and key in cache:
        return cache[key]["best"], cache[key]["timings"]
    timings = {}
    best, best_ms = None, float("inf")
    for cfg in candidates or (CANDIDATES + selection_candidates(slot_capacity)):
        ms = time_config(setup, prim, ids, precision, cfg, repeats, slot_capacity, device)
        timings[json.dumps(cfg, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = cfg, ms
    cache[key] = {"best": best, "timings": timings}
    try:  # atomic replace: ranks of a multi-GPU run may write at once
        tmp = f"{CACHE}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, CACHE)
    except OSError:
        pass
    return best, timings


def sample_ids(n, k, seed=0):
    """k event indices of n, sorted (for tuning on a sample)."""
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False))
