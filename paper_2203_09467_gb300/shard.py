"""Event sharding across ranks (one process per GPU).

Events are independent (the paper's domain replication: events are
decomposed across MPI ranks, Sec. 2.1), so a multi-GPU run partitions the
events, transports each shard on its own GPU with no exchange while
stepping, and gathers the per-event results once at the end.
"""
from __future__ import annotations

import heapq

import numpy as np


def event_costs(prim, n_events):
    """Cost of each event: the sum of its primaries' kinetic energies (the
    number of track-steps of a shower grows about linearly with it)."""
    return np.bincount(np.asarray(prim["event"]), weights=np.asarray(prim["T"], float), minlength=n_events)


def partition_by_cost(costs, world):
    """Greedy longest-processing-time partition: events in decreasing cost,
    each to the currently least-loaded rank.  Returns one sorted index array
    per rank."""
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    for e in np.argsort(-np.asarray(costs, float), kind="stable"):
        load, r = heapq.heappop(heap)
        parts[r].append(int(e))
        heapq.heappush(heap, (load + float(costs[e]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def shard_primaries(prim, events):
    """Primaries of the listed events, renumbered 0..len(events)-1 in order."""
    events = np.asarray(events, np.int64)
    ev = np.asarray(prim["event"])
    remap = -np.ones(int(ev.max()) + 1 if len(ev) else 0, np.int64)
    remap[events] = np.arange(len(events))
    keep = np.isin(ev, events)
    out = {k: np.asarray(v)[keep] for k, v in prim.items()}
    out["event"] = remap[out["event"]].astype(np.int32)
    order = np.argsort(out["event"], kind="stable")
    return {k: v[order] for k, v in out.items()}


def local_shard(prim, event_ids, rank, world):
    """This rank's events of one workload (cost-balanced partition): the
    original event indices, their primaries (renumbered) and their ids."""
    n = len(event_ids)
    mine = partition_by_cost(event_costs(prim, n), world)[rank]
    return mine, shard_primaries(prim, mine), np.asarray(event_ids)[mine]


def gather_events(mine, hist, summ, n_events, world, group=None):
    """The one gather of a sharded run: every rank's per-event results,
    placed in the original event order on every rank.  With world == 1 no
    collective is used."""
    if world == 1:
        return hist, summ
    import torch.distributed as dist
    gathered = [None] * world
    dist.all_gather_object(gathered, (np.asarray(mine), np.asarray(hist), np.asarray(summ)), group=group)
    H = np.zeros((n_events, np.asarray(hist).shape[1]))
    S = np.zeros((n_events, np.asarray(summ).shape[1]))
    for idx, h, s in gathered:
        H[idx] = h
        S[idx] = s
    return H, S


def run_sharded(engine, prim, event_ids, rank, world, group=None):
    """Transport this rank's shard with engine(prim, ids) -> (hist, summary)
    and gather every rank's results on every rank, in the original event
    order.  With world == 1 no collective is used."""
    mine, p, ids = local_shard(prim, event_ids, rank, world)
    hist, summ = engine(p, ids)
    return gather_events(mine, hist, summ, len(event_ids), world, group)
