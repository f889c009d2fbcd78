"""Host-side logic of the multi-GPU runs: independent boxes shared out over ranks (no data exchange
between boxes, so no collective on the data path) and the timing reduction of the benchmark."""
from __future__ import annotations


def shard_boxes(box_sizes, world: int) -> list:
    """Greedy longest-processing-time assignment of independent boxes to `world` ranks: boxes in
    descending size, each to the currently lightest rank (ties: lowest rank).  Returns, per rank,
    the list of box indices in ascending order.  Deterministic, so every rank computes the same
    plan without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    owned = [[] for _ in range(world)]
    order = sorted(range(len(box_sizes)), key=lambda b: (-int(box_sizes[b]), b))
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(b)
        load[r] += int(box_sizes[b])
    return [sorted(o) for o in owned]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (the step time of a weak-scaling run); identity without a
    process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """Sum over ranks (particles processed by the whole job)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


ENSEMBLE_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h")


def ensemble_shard(boxes, world: int = 1, rank: int = 0) -> dict:
    """This rank's part of an ensemble of independent boxes (dicts of per-particle arrays with "n",
    "mass" and "gamma"), as the arguments of a batch context: the boxes shard_boxes assigns to the
    rank, in ascending box order, concatenated.  Returns {"boxes": box indices, "offsets":
    int64[k+1], "mass": float64[k], "gamma": float64[k], "state": concatenated arrays}."""
    import numpy as np
    plan = shard_boxes([b["n"] for b in boxes], world)[rank]
    mine = [boxes[b] for b in plan]
    off = np.concatenate([[0], np.cumsum([b["n"] for b in mine])]).astype(np.int64)
    state = {k: np.concatenate([b[k] for b in mine]) if mine else np.zeros(0) for k in ENSEMBLE_FIELDS}
    state["mass"] = 1.0
    return {"boxes": plan, "offsets": off, "mass": np.array([b["mass"] for b in mine], dtype=np.float64),
            "gamma": np.array([b["gamma"] for b in mine], dtype=np.float64), "state": state}
