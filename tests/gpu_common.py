"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def to_orig(values, ids):
    """Scatter per-particle values given in the library's (Morton) order back to the original order."""
    out = np.empty_like(values)
    out[ids.astype(np.int64)] = values
    return out


def random_positions(n, seed, kind="uniform"):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        p = rng.uniform(0, 1, size=(3, n))
    elif kind == "cluster":
        p = np.mod(0.5 + 0.08 * rng.standard_normal(size=(3, n)), 1.0)
    elif kind == "dups":
        base = rng.uniform(0, 1, size=(3, n // 3 + 1))
        p = base[:, rng.integers(0, base.shape[1], size=n)]
    else:
        raise ValueError(kind)
    return p[0].copy(), p[1].copy(), p[2].copy()
