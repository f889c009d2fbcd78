"""Seeded synthetic initial conditions for the SPH workloads (periodic unit box).

This module only builds inputs: particle positions on a jittered cubic lattice, Gaussian velocities,
internal energy and a first smoothing-length guess.  It holds none of the method's arithmetic (no
kernel sums, no neighbour search, no integration) and is the one module that both the CUDA path's
tests and the CPU oracle's tests draw their inputs from.

Recipes (numpy PCG64; seed = 12345 + workload index unless given):
  * ``lattice``: n^3 particles at ((i,j,k)+0.5)/n, each coordinate jittered by U(-j dx, +j dx) with
    j = 0.01 (dx = 1/n), velocities N(0, sigma^2) per component, u = u0, m = 1/N, h = hfact dx.
  * ``sedov``: the same lattice with v = 0 and background u = 1e-8; energy E = 1 is added to the
    particles within 2 h0 of the box centre, weighted by a cubic B-spline bump of radius 2 h0 and
    normalised so that sum_i m du_i = E exactly.  This stands in for the paper's Sedov-Taylor
    set-up (Sect. 4.4 and Sect. 5.1.2) on a cubic instead of a close-packed lattice.
  * ``ensemble``: independent boxes with N_b = round(exp(U(ln 2048, ln 262144))), side
    round(N_b^(1/3)), sigma ~ U[0.01, 0.3], gamma in {5/3, 7/5}; box b uses seed + 1000 b.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h")


def lattice(n_side: int, sigma_v: float = 0.01, u0: float = 1.0, jitter: float = 0.01, hfact: float = 1.2,
            seed: int = 12345) -> dict:
    """Jittered cubic lattice in the periodic unit box."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_side ** 3
    dx = 1.0 / n_side
    idx = np.arange(n_side, dtype=np.float64)
    gx, gy, gz = np.meshgrid(idx, idx, idx, indexing="ij")
    pos = [(g.reshape(-1) + 0.5) * dx for g in (gx, gy, gz)]
    out = {}
    for name, p in zip(("x", "y", "z"), pos):
        q = p + rng.uniform(-jitter * dx, jitter * dx, size=n)
        q = np.where(q >= 1.0, q - 1.0, q)
        q = np.where(q < 0.0, q + 1.0, q)
        out[name] = q
    for name in ("vx", "vy", "vz"):
        out[name] = rng.normal(0.0, sigma_v, size=n) if sigma_v > 0 else np.zeros(n)
    out["u"] = np.full(n, float(u0))
    out["h"] = np.full(n, hfact * dx)
    out["mass"] = 1.0 / n
    out["n"] = n
    out["dx"] = dx
    return out


def _bump(q: np.ndarray) -> np.ndarray:
    """Cubic B-spline bump on [0, 2) used only to spread the Sedov energy (unnormalised)."""
    w = np.zeros_like(q)
    a = q < 1.0
    b = (q >= 1.0) & (q < 2.0)
    w[a] = 1.0 - 1.5 * q[a] ** 2 + 0.75 * q[a] ** 3
    w[b] = 0.25 * (2.0 - q[b]) ** 3
    return w


def sedov(n_side: int, energy: float = 1.0, u_bg: float = 1e-8, jitter: float = 0.01, hfact: float = 1.2,
          seed: int = 12346) -> dict:
    """Sedov-Taylor blast in the periodic unit box: background rho = 1, u = u_bg, v = 0."""
    s = lattice(n_side, sigma_v=0.0, u0=u_bg, jitter=jitter, hfact=hfact, seed=seed)
    h0 = hfact * s["dx"]
    r = np.sqrt((s["x"] - 0.5) ** 2 + (s["y"] - 0.5) ** 2 + (s["z"] - 0.5) ** 2)
    w = _bump(r / h0)
    tot = s["mass"] * w.sum()
    s["u"] = s["u"] + energy * w / tot
    return s


def ensemble(n_boxes: int = 256, seed: int = 12349, n_min: int = 2048, n_max: int = 262144) -> list:
    """Independent periodic boxes of log-uniform size (see module docstring)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = np.round(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_boxes))).astype(np.int64)
    sides = np.maximum(np.round(np.cbrt(nb)).astype(np.int64), 2)
    sigmas = rng.uniform(0.01, 0.3, size=n_boxes)
    gammas = np.where(rng.uniform(size=n_boxes) < 0.5, 5.0 / 3.0, 7.0 / 5.0)
    boxes = []
    for b in range(n_boxes):
        s = lattice(int(sides[b]), sigma_v=float(sigmas[b]), seed=seed + 1000 * (b + 1))
        s["gamma"] = float(gammas[b])
        s["n_drawn"] = int(nb[b])
        boxes.append(s)
    return boxes


def perfect_lattice(n_side: int, hfact: float = 1.2, h_scale: float = 1.0) -> dict:
    """Unjittered cubic lattice, v = 0, u = 1 (used by the lattice pins)."""
    s = lattice(n_side, sigma_v=0.0, u0=1.0, jitter=0.0, hfact=hfact)
    s["h"] = s["h"] * h_scale
    return s
