"""Multi-rank host logic on CPU: box sharding and the benchmark's reductions over 2 gloo ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_boxes_balanced_and_complete():
    from paper_2503_09713_gb300 import replicas, workloads
    import numpy as np
    rng = np.random.default_rng(0)
    sizes = np.round(np.exp(rng.uniform(np.log(2048), np.log(262144), size=256))).astype(int)
    for world in (1, 2, 3, 8):
        plan = replicas.shard_boxes(sizes, world)
        flat = sorted(b for o in plan for b in o)
        assert flat == list(range(256))
        loads = [sum(sizes[b] for b in o) for o in plan]
        assert max(loads) - min(loads) <= sizes.max()     # LPT bound
    assert replicas.shard_boxes([5, 1, 1], 2) == [[0], [1, 2]]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2503_09713_gb300 import replicas
    m = replicas.max_over_ranks(10.0 + rank, dist)
    s = replicas.sum_over_ranks(1000 * (rank + 1), dist)
    plan = replicas.shard_boxes([7, 3, 5, 1, 9, 2], world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, s, plan))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [3000.0, 3000.0]
    assert res[0][3] == res[1][3]


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2503_09713_gb300 import replicas, workloads
    boxes = workloads.ensemble(24, seed=12349, n_max=20000)
    part = replicas.ensemble_shard(boxes, world, rank)
    n_local = int(part["offsets"][-1])
    n_total = replicas.sum_over_ranks(n_local, dist)
    # each rank's boxes, as the per-box slices of its concatenated state
    mine = {}
    for k, b in enumerate(part["boxes"]):
        lo, hi = part["offsets"][k], part["offsets"][k + 1]
        mine[b] = {f: part["state"][f][lo:hi].copy() for f in ("x", "vx", "u", "h")}
        mine[b]["mass"] = part["mass"][k]
        mine[b]["gamma"] = part["gamma"][k]
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, part["boxes"], n_local, n_total, mine))


def test_ensemble_shard_two_gloo_ranks():
    """The ensemble split over 2 ranks: the shards are disjoint and together hold every box once,
    each box arrives with the same particles, mass and gamma as in the single-rank ensemble, and
    the particle count summed over ranks is the whole ensemble's."""
    import numpy as np
    import torch.multiprocessing as mp
    from paper_2503_09713_gb300 import replicas, workloads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    boxes = workloads.ensemble(24, seed=12349, n_max=20000)
    full = replicas.ensemble_shard(boxes, 1, 0)
    assert full["boxes"] == list(range(24))
    b0, b1 = set(res[0][1]), set(res[1][1])
    assert not (b0 & b1) and (b0 | b1) == set(range(24))
    total = int(full["offsets"][-1])
    assert res[0][3] == res[1][3] == total == res[0][2] + res[1][2]
    for _, _, _, _, mine in res:
        for b, got in mine.items():
            lo, hi = full["offsets"][b], full["offsets"][b + 1]
            for f in ("x", "vx", "u", "h"):
                assert np.array_equal(got[f], full["state"][f][lo:hi]), (b, f)
            assert got["mass"] == full["mass"][b] and got["gamma"] == full["gamma"][b]
