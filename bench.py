"""Benchmark of the EM transport loop on GB300 (one JSON line on rank 0).

A benchmark step is one complete pass of the transport hot path over one
batch: submit every event of the workload, step until no track is left,
read every event's scores.  Default workload: the sampling calorimeter
(50 x (2 mm Pb + 5 mm LAr), 10,000 events of one 10 GeV electron, FP64).

  value : track-steps/s with the primaries already in device memory when the
          timed region starts (CUDA events on the library's stream)
  e2e   : the same through host buffers (pinned), host<->device copies of the
          primaries and of all scores inside the timed region
  roofline : the step kernel (dominant by time): algorithmic track-state
          bytes per launch / mean launch duration (CUDA events around each
          launch, recorded by the library on its stream)
  cpu_baseline : the FP64 CPU oracle on the host cores, on a bounded sample
          of the same workload

Under torchrun with N ranks the workload is one set of N x events events,
partitioned across the ranks by cost (greedy on the primaries' energy,
paper_2203_09467_gb300.shard): each rank transports its shard with no
exchange while stepping (weak scaling: the per-GPU work stays fixed), and
the per-event results are gathered once, in event order, after the timed
steps.  `--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_09467_gb300 import workloads as W  # noqa: E402

METRIC = "track-steps/s"

# DRAM traffic per track-step of the step kernels (dram__bytes_read.sum +
# dram__bytes_write.sum from ncu captures of four launches of one step
# kernel on a smaller run of the same workload, divided by the tracks those
# launches stepped; summary and commands in profiles/), per workload,
# precision and step schedule.  Reported only while the kernel sources are
# the ones that were measured (SHA-256 below).
TRAFFIC = {
    "kernel_sha256": "15abf5842738ce5d4e9c433fb3bef2edc32a6368716462450f708d34bdded67d",
    "bytes_per_track_step": {"calo/fp64/pipelined": 101.6, "calo/fp64/split": 114.4, "calo/mixed/pipelined": 97.5,
                             "calo_field/fp64/split": 109.1},
    "source": "profiles/step_kernels_dram_traffic.md",
}
# Algorithmic FP64 work of one track-step of the method, fixed by its
# definition: a census of the FP64 operations of the oracle's step on the
# workload (oracle/census.py; summary in profiles/fp64_census_of_the_step.md),
# in flops with add, sub, mul, div and sqrt one each and an fma two
# (comparisons and elementary functions are listed there, not counted).  It
# does not change when the kernels are optimised.
FLOPS_PER_TRACK_STEP = {"calo": 43.09, "calo_field": 967.93, "cms": 73.49, "slab": 59.05, "batched": 969.84}
# nominal FP64 peak of GB300: 152 SMs x 2 DFMA per clock x 2 flops x 2.06 GHz
FP64_NOMINAL_GFLOPS = 1252.5
KERNEL_SOURCES = ["emt_device.cuh", "emt_intdiv.cuh", "emt_intlog.cuh", "emt_logtab.h", "emt_step.cuh",
                  "emt_split.cuh", "emt_launch.cuh", "emt_kernels_fp64.cu", "emt_kernels_fp64_persist.cu",
                  "emt_kernels_fp64_split.cu", "emt_kernels_fp64_pipe.cu", "emt_kernels_mixed.cu",
                  "emt_kernels_mixed_persist.cu", "emt_kernels_mixed_split.cu", "emt_kernels_mixed_pipe.cu"]


def kernel_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2203_09467_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def workload(name, n_events):
    """Setup, primaries and event ids of the whole workload."""
    if name == "calo":
        s = W.calo_setup()
        prim = W.calo_primaries(n_events, seed=s.seed)
        desc = f"sampling calorimeter 50x(2mm Pb+5mm LAr), {n_events} events x 10 GeV e-"
    elif name == "slab":
        s = W.slab_setup()
        prim = W.slab_primaries(n_events)
        desc = f"5 cm Pb slab, {n_events} events x 100 MeV e-"
    elif name == "calo_field":
        s = W.calo_field_setup()
        prim = W.calo_field_primaries(n_events, seed=s.seed)
        desc = f"calorimeter in 2 T field, {n_events} events, e-/e+/gamma 1-100 GeV"
    elif name == "batched":
        s = W.calo_field_setup()
        s.seed = 4
        prim = W.batched_primaries(n_events, seed=4)
        desc = f"calorimeter in 2 T field, {n_events} events of 1-64 primaries, 0.1-100 GeV"
    elif name == "served":
        s = W.calo_field_setup()
        s.seed = 5
        prim = W.served_primaries(n_events, seed=5)
        desc = f"calorimeter in 2 T field, {n_events} requests of 1-100 primaries, 1-50 GeV"
    elif name in ("cms", "cms_field"):
        s = W.cms_setup() if name == "cms" else W.cms_field_setup()
        prim = W.cms_primaries(n_events, 1000, seed=s.seed)
        desc = (f"CMS-like 6 cylindrical shells to 375 cm (vacuum, Si, Pb, C, Ti, Fe)"
                f"{', 3.8 T along z' if name == 'cms_field' else ''}, {n_events} events x 1000 isotropic 1 GeV photons")
    else:
        raise SystemExit(f"unknown workload {name}")
    ids = np.arange(n_events, dtype=np.uint64)
    return s, prim, ids, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            # nvidia-smi takes a moment to start: wait (at most 3 s) for its
            # first sample so that the samples cover the timed region
            t0 = time.monotonic()
            while os.path.getsize(self.path) == 0 and time.monotonic() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(setup, prim, ids, budget_s=12.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample
    of the workload (events in order until ~budget_s of work)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    orc = oracle.Oracle(setup.materials, setup.physics, setup.layers, setup.world, setup.seed)
    n_total = len(ids)
    n = min(n_total, max(cores * 4, 64))
    steps = 0.0
    t = 0.0
    done = 0
    while done < n_total:
        take = min(n, n_total - done)
        sub = W.subset(prim, np.arange(done, done + take))
        t0 = time.perf_counter()
        _, summ = orc.run(sub, take, ids[done:done + take], n_threads=cores)
        t += time.perf_counter() - t0
        steps += summ[:, 4].sum()
        done += take
        if t > budget_s:
            break
        n = min(n_total - done, int(take * max(1.0, min(4.0, budget_s / max(t, 1e-3) / 2)))) or 1
    # one core: the first events of the workload for about a quarter of the budget
    t1, steps1, done1 = 0.0, 0.0, 0
    while done1 < n_total and t1 < budget_s / 4:
        take = min(max(1, cores), n_total - done1)
        sub = W.subset(prim, np.arange(done1, done1 + take))
        t0 = time.perf_counter()
        _, summ = orc.run(sub, take, ids[done1:done1 + take], n_threads=1)
        t1 += time.perf_counter() - t0
        steps1 += summ[:, 4].sum()
        done1 += take
    orc.close()
    return {"value": steps / t, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"first {done} of {n_total} events of the workload, {int(steps)} track-steps, "
                      f"{t:.1f} s on {cores} threads",
            "value_1core": steps1 / t1,
            "sample_1core": f"first {done1} events, {int(steps1)} track-steps, {t1:.1f} s on 1 thread"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    setup, prim, ids, desc = workload(args.workload, args.events)
    import oracle
    cores = len(os.sched_getaffinity(0))
    orc = oracle.Oracle(setup.materials, setup.physics, setup.layers, setup.world, setup.seed)
    # each step: a bounded sample of the workload (sized for a few seconds)
    n = min(args.events, args.ref_events)
    sub = W.subset(prim, np.arange(n))
    for _ in range(args.warmup):
        orc.run(sub, n, ids[:n], n_threads=cores)
    t = 0.0
    steps = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, summ = orc.run(sub, n, ids[:n], n_threads=cores)
        t += time.perf_counter() - t0
        steps += summ[:, 4].sum()
    v = steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "sample_events_per_step": n},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"first {n} events of the workload per step"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2203_09467_gb300 import emt
    from paper_2203_09467_gb300 import shard

    # one workload of world x events events, partitioned across the ranks
    n_total = args.events * world
    setup, prim_all, ids_all, desc = workload(args.workload, n_total)
    mine, prim, ids = shard.local_shard(prim_all, ids_all, rank, world)
    n = len(ids)
    tune = None
    if args.loop == "auto":
        from paper_2203_09467_gb300 import autotune
        best, timings = autotune.autotune(args.workload, setup, prim, ids, args.precision, use_cache=not args.retune,
                                          slot_capacity=args.slots, device=local)
        cfg = dict(best)
        tune = {"best": best, "ms_per_candidate": timings}
    else:
        cfg = {"block_size": args.block, "loop_mode": args.loop, "graph_steps": args.graph_steps,
               "schedule": args.schedule}
    ctx = emt.context_for(setup, device=local, precision=args.precision, slot_capacity=args.slots, max_events=n,
                          **cfg)
    stream = ctx.stream
    dev = torch.device("cuda", local)
    dprim = {k: torch.as_tensor(v).to(dev) for k, v in prim.items()}
    nb = setup.n_bins
    hist_d = torch.empty((n, nb), dtype=torch.float64, device=dev)
    summ_d = torch.empty((n, 6), dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    pin = {k: torch.as_tensor(v).pin_memory() for k, v in prim.items()}
    hist_h = torch.empty((n, nb), dtype=torch.float64).pin_memory()
    summ_h = torch.empty((n, 6), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1)

    def step_device():
        ctx.submit(ids, dprim)
        st = ctx.run()
        ctx.read_all(hist_d, summ_d)
        return st

    def step_host():
        ctx.submit(ids, {k: v.numpy() for k, v in pin.items()})
        st = ctx.run()
        ctx.read_all(hist_h.numpy(), summ_h.numpy())
        return st

    for _ in range(args.warmup):
        flush_l2()
        step_device()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = []
    stats = []
    launches = 0
    for _ in range(args.steps):
        flush_l2()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = step_device()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        stats.append(st)
        launches += st["kernel_launches"] + 6  # + admission (5 kernels) and gather
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(sum(ms))
    steps_done = float(sum(s["track_steps"] for s in stats))
    if world > 1:
        t = torch.tensor([total_ms, steps_done], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
        total_ms_all, steps_all = float(tmax[0]), float(t[1])
    else:
        total_ms_all, steps_all = total_ms, steps_done
    value = steps_all / (total_ms_all / 1e3)

    # end to end through host buffers
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        flush_l2()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = step_host()
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_steps = st["track_steps"]
    e2e_value = e2e_steps * world / (max(e2e_ms) / 1e3) if world == 1 else None
    if world > 1:
        t = torch.tensor([max(e2e_ms), float(e2e_steps)], dtype=torch.float64, device=dev)
        dist.all_reduce(t[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
        e2e_value = float(t[1]) / (float(t[0]) / 1e3)
    h2d = sum(v.numel() * v.element_size() for v in pin.values()) + ids.nbytes
    d2h = hist_h.numel() * 8 + summ_h.numel() * 8

    # the one gather of the sharded run: every event's results in event
    # order (after the timed steps; no collective while stepping)
    H, S = shard.gather_events(mine, hist_h.numpy(), summ_h.numpy(), n_total, world)
    gather = {"events": int(len(S)), "events_with_deposit": int((S[:, 0] > 0).sum()),
              "max_ledger_error": float(np.max(np.abs(S[:, 3] - S[:, 0] - S[:, 1] - S[:, 2]) / S[:, 3]))}

    # roofline of the step kernel
    dfma = emt.measure_dfma_rate(local)  # FP64 FMAs per second, measured now on this GPU
    # FP64 divisions and logarithms per second, native and on the integer pipe
    op_rates = emt.measure_fp64_op_rates(local)
    peaks, src = load_peaks()
    kern_ms = sum(s["kernel_ms"] for s in stats)
    kern_launch = sum(s["iterations"] for s in stats)  # one step-loop iteration = one step (1 or 2 kernels)
    state_bytes = sum(s["state_bytes"] for s in stats)
    achieved = state_bytes / (kern_ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "peak_source": f"{src} hbm_gbs",
            "kernel": {"split": "step = k_transport + k_interact",
                       "pipelined": "step = k_pipe"}.get(cfg.get("schedule"), "k_step"),
            "launches": kern_launch, "mean_launch_ms": kern_ms / max(kern_launch, 1),
            "algorithmic_bytes_per_launch": state_bytes / max(kern_launch, 1),
            "kernel_share_of_step": kern_ms / total_ms}
    key = f"{args.workload}/{args.precision}/{cfg.get('schedule', 'fused')}"
    current = TRAFFIC["kernel_sha256"] == kernel_sha256()
    per_step = TRAFFIC["bytes_per_track_step"].get(key) if current else None
    steps_per_launch = steps_done / max(kern_launch, 1)
    if args.traffic_per_launch:
        roof["traffic"] = args.traffic_per_launch
    elif per_step:
        roof["traffic"] = per_step * steps_per_launch
        roof["traffic_source"] = (f"{TRAFFIC['source']}: {per_step:.1f} B per track-step x "
                                  f"{steps_per_launch:.0f} track-steps per launch")
    flops = FLOPS_PER_TRACK_STEP.get(args.workload)
    roof_hbm = None
    if flops and args.precision == "fp64":
        # the FP64 step kernels are led by the FP64 pipe: report the
        # arithmetic roofline (algorithmic flops per track-step from the
        # census of the method), and the HBM one beside it
        roof_hbm = roof
        ach = flops * steps_done / (kern_ms / 1e3) / 1e9
        peak_f = 2.0 * dfma / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": peak_f, "unit": "GFLOP/s",
                "frac": ach / peak_f, "traffic": roof_hbm["traffic"],
                "peak_source": f"measured now: {dfma / 1e9:.1f} G DFMA/s (emt_measure_dfma_rate, independent "
                               "chains) x 2 flops",
                "frac_of_nominal": ach / FP64_NOMINAL_GFLOPS, "peak_nominal": FP64_NOMINAL_GFLOPS,
                "kernel": roof_hbm["kernel"], "launches": kern_launch,
                "mean_launch_ms": kern_ms / max(kern_launch, 1),
                "algorithmic_flops_per_launch": flops * steps_per_launch,
                "flops_per_track_step": flops,
                "flops_source": "census of the oracle's step (oracle/census.py)",
                "kernel_share_of_step": kern_ms / total_ms}

    # the plain form: the same events submitted and run one at a time, with
    # a host-driven step loop (one launch per step: the fused schedule suits
    # a single event best) and with the persistent step loop
    forms = None
    if args.one_at_a_time > 0 and rank == 0:
        k = min(args.one_at_a_time, n)
        # primaries of event e: [first[e], first[e + 1]) (grouped by event)
        first = np.searchsorted(prim["event"], np.arange(n + 1))
        forms = {"batched": {"events_per_s": n / (total_ms / 1e3 / args.steps), "track_steps_per_s": value / world,
                             "config": cfg}}
        for name, loop in (("one_at_a_time", dict(loop_mode="plain")),
                           ("one_at_a_time_persistent", dict(loop_mode="persistent", graph_steps=256))):
            single = emt.context_for(setup, device=local, precision=args.precision, slot_capacity=1 << 22,
                                     max_events=1, block_size=cfg["block_size"], schedule="fused", **loop)
            steps1 = 0
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(single.stream)
            for e in range(k):
                lo, hi = int(first[e]), int(first[e + 1])
                sub = {kk: v[lo:hi] for kk, v in dprim.items()}
                sub["event"] = torch.zeros(hi - lo, dtype=torch.int32, device=dev)
                single.submit(ids[e:e + 1], sub)
                steps1 += single.run()["track_steps"]
                single.read_all(hist_d[e:e + 1], summ_d[e:e + 1])
            b.record(single.stream)
            b.synchronize()
            t1 = a.elapsed_time(b) / 1e3
            single.close()
            forms[name] = {"events_per_s": k / t1, "track_steps_per_s": steps1 / t1, "sample_events": k,
                           "loop": loop["loop_mode"]}

    ctx.close()
    if args.diagnostics and rank == 0:
        diagnostics(args, emt, setup, prim, ids, cfg, local)
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": desc, "precision": args.precision, "schedule": cfg.get("schedule", "fused"),
                   "loop": cfg["loop_mode"],
                   "graph_steps": cfg["graph_steps"], "block": cfg["block_size"] or 256,
                   "track_selection": {k: cfg[k] for k in ("max_active", "select", "spill_above") if k in cfg} or None,
                   "slot_capacity": args.slots, "events_per_gpu": n, "events_total": n_total,
                   "partition": "one workload split across the GPUs by cost (greedy on primary energy)",
                   "l2": "512 MB buffer written between timed steps; track state >> L2"},
        "events_per_s": n * world / (total_ms_all / 1e3 / args.steps),
        "iterations_per_step": stats[0]["iterations"], "peak_tracks": max(s["peak_tracks"] for s in stats),
        # per timed step: steps deferred for want of a slot, tracks moved to
        # host memory and back, tracks held by the selection, RK4 substeps
        "run_stats_per_step": {k: sum(s[k] for s in stats) / len(stats)
                               for k in ("deferred", "spilled", "held", "rk4_substeps")},
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "gather": gather,
        "roofline": roof,
        "fp64_op_rates": op_rates,
        "clocks": clk,
    }
    if roof_hbm:
        line["roofline_hbm"] = roof_hbm
    if forms:
        line["forms"] = forms
    if tune:
        line["autotune"] = tune
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(setup, prim, ids, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def diagnostics(args, emt, setup, prim, ids, cfg, device):
    """Sec. 3.2's diagnostics of one untimed run of the workload: tracks in
    flight, interactions, deferred and held copies and device time per step
    (plain driver), and the steps-per-track histogram by particle type."""
    nb = 4096
    ctx = emt.context_for(setup, device=device, precision=args.precision, slot_capacity=args.slots,
                          max_events=len(ids), block_size=cfg["block_size"], schedule=cfg.get("schedule", "split"),
                          step_hist_bins=nb)
    ctx.submit(ids, prim)
    st, rec = ctx.run_traced()
    ctx.read_all()
    sh = ctx.read_step_hist()
    ctx.close()
    out = {"workload": args.workload, "precision": args.precision, "stats": st,
           "records": {"photons": rec[:, 0].tolist(), "charged": rec[:, 1].tolist(),
                       "interacting": rec[:, 2].tolist(), "deferred": rec[:, 3].tolist(),
                       "held": rec[:, 4].tolist(), "ms": rec[:, 5].tolist()},
           "steps_per_track": {"gamma": sh[0].tolist(), "electron": sh[1].tolist(), "positron": sh[2].tolist()}}
    with open(args.diagnostics, "w") as f:
        json.dump(out, f)


def served_arm(args):
    """Event requests arriving as a Poisson process at each rate; continuous
    batching against the one-batch-at-a-time schedule on the same GPU.
    Latency = completion - arrival (host monotonic clock)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2203_09467_gb300 import emt

    setup = W.calo_field_setup()
    setup.seed = 5
    rates = [float(r) for r in args.rates.split(",")]
    results = []
    loops = args.serve_loops.split(",")
    for ri, rate in enumerate(rates):
        arrival = W.poisson_arrivals(rate, args.duration, seed=5 + ri)
        n = len(arrival)
        prim = W.served_primaries(n, seed=5 + ri)
        ids = np.arange(n, dtype=np.uint64) + np.uint64(1_000_000 * ri)
        row = {"rate_hz": rate, "requests": n, "duration_s": args.duration}
        for loop in loops:
            for mode in ("continuous", "batch"):
                # the graph driver replays 6 steps per launch; the persistent
                # loop runs up to 6 steps per launch (or fewer, ending early)
                ctx = emt.context_for(setup, precision=args.precision, slot_capacity=args.serve_slots,
                                      max_events=args.serve_events, loop_mode=loop, graph_steps=6,
                                      schedule="fused" if loop == "persistent" else "split")
                admit, done, hist, summ = ctx.serve(ids, arrival, prim, mode=mode, steps_per_poll=6)
                ctx.close()
                lat = done - arrival
                span = done.max() - arrival.min()
                key = mode if loop == "graph" else f"{mode}_{loop}"
                row[key] = {"events_per_s": n / span, "p50_latency_s": float(np.percentile(lat, 50)),
                            "p99_latency_s": float(np.percentile(lat, 99)),
                            "mean_queue_s": float(np.mean(admit - arrival)),
                            "track_steps": float(summ[:, 4].sum()), "loop": loop}
        results.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    top = results[-1]
    line = {"metric": "events/s", "value": top["continuous"]["events_per_s"], "unit": "events/s", "n_gpus": 1,
            "steps": len(rates), "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "served: Poisson requests of 1-100 primaries (e-/e+/gamma, 1-50 GeV) on the "
                                   "calorimeter in a 2 T field", "precision": args.precision,
                       "track_slots": args.serve_slots, "event_slots": args.serve_events},
            "rates": results}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="emt", choices=["emt", "reference"])
    ap.add_argument("--workload", default="calo",
                    choices=["calo", "slab", "calo_field", "batched", "served", "cms", "cms_field"])
    ap.add_argument("--rates", default="10,100,1000", help="served: request rates (Hz)")
    ap.add_argument("--duration", type=float, default=60.0, help="served: seconds of requests per rate")
    ap.add_argument("--serve-slots", type=int, default=1 << 22, help="served: track-slot pool")
    ap.add_argument("--serve-events", type=int, default=4096, help="served: event slots")
    ap.add_argument("--serve-loops", default="graph,persistent",
                    help="served: step-loop drivers to compare (graph, persistent, plain)")
    ap.add_argument("--events", type=int, default=None, help="default 10,000 (100 for cms, cms_field)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--loop", default="auto", choices=["auto", "plain", "graph", "persistent"],
                    help="auto: autotune block size and loop driver on the workload first")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--graph-steps", type=int, default=12)
    ap.add_argument("--slots", type=int, default=1 << 25)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--schedule", default="split", choices=["fused", "split", "pipelined"],
                    help="step schedule when --loop is not auto")
    ap.add_argument("--one-at-a-time", type=int, default=100,
                    help="events of the plain one-event-at-a-time form to time (0: skip)")
    ap.add_argument("--ref-events", type=int, default=1000)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--diagnostics", default=None,
                    help="write per-step records and the steps-per-track histogram of one untimed run (JSON)")
    ap.add_argument("--traffic-per-launch", type=float, default=None,
                    help="DRAM bytes per step-kernel launch from an ncu capture of this kernel")
    args = ap.parse_args()
    if args.events is None:
        args.events = 100 if args.workload in ("cms", "cms_field") else 10000
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "served":
        served_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
