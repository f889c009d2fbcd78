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
