"""Multi-rank host logic on the CPU: two gloo ranks each transport a
cost-balanced shard of the events (the FP64 oracle stands in for the
per-GPU engine) and the gathered per-event results equal one
single-process run, bit for bit."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2203_09467_gb300 import shard
from paper_2203_09467_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup(n=24):
    s = W.calo_setup()
    prim = W.multi_primaries(n, 1, 5, 200.0, 20.0, seed=41)
    ids = np.arange(100, 100 + n, dtype=np.uint64)
    return s, prim, ids


def _engine(s):
    import oracle
    o = oracle.Oracle(s.materials, s.physics, s.layers, s.world, s.seed)
    return lambda prim, ids: o.run(prim, len(ids), ids, n_threads=2)


def _worker(rank, world, port, out_dir, n=24):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, prim, ids = _setup(n)
    H, S = shard.run_sharded(_engine(s), prim, ids, rank, world)
    np.save(os.path.join(out_dir, f"h{rank}.npy"), H)
    np.save(os.path.join(out_dir, f"s{rank}.npy"), S)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_balances_cost():
    costs = np.random.default_rng(0).lognormal(size=1000)
    parts = shard.partition_by_cost(costs, 4)
    assert sorted(np.concatenate(parts).tolist()) == list(range(1000))
    loads = [costs[p].sum() for p in parts]
    assert max(loads) / min(loads) < 1.01


def test_two_gloo_ranks_equal_single_run(tmp_path):
    import oracle
    oracle.build()  # once, before the ranks start
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    s, prim, ids = _setup()
    H1, S1 = shard.run_sharded(_engine(s), prim, ids, 0, 1)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"h{r}.npy"), H1)
        assert np.array_equal(np.load(tmp_path / f"s{r}.npy"), S1)


def test_rank_without_events(tmp_path):
    """Three gloo ranks and two events: one rank's shard is empty, and the
    gathered results still equal the single-process run."""
    import oracle
    oracle.build()
    world, n = 3, 2
    assert min(len(p) for p in shard.partition_by_cost(shard.event_costs(_setup(n)[1], n), world)) == 0
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), n), nprocs=world, join=True)
    s, prim, ids = _setup(n)
    H1, S1 = shard.run_sharded(_engine(s), prim, ids, 0, 1)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"h{r}.npy"), H1)
        assert np.array_equal(np.load(tmp_path / f"s{r}.npy"), S1)


def test_local_shards_cover_one_workload_once():
    """The benchmark's split of one workload: the ranks' shards are disjoint,
    cover every event, keep each event's primaries together and in order,
    and carry near-equal primary energy."""
    s, prim, ids = _setup(n=400)
    world = 4
    seen = []
    loads = []
    for r in range(world):
        mine, p, local_ids = shard.local_shard(prim, ids, r, world)
        seen.extend(mine.tolist())
        assert np.array_equal(local_ids, ids[mine])
        assert np.array_equal(np.unique(p["event"]), np.arange(len(mine)))
        for k, e in enumerate(mine[:20]):
            want = prim["T"][prim["event"] == e]
            assert np.array_equal(p["T"][p["event"] == k], want)
        loads.append(p["T"].sum())
    assert sorted(seen) == list(range(400))
    assert max(loads) / min(loads) < 1.02
