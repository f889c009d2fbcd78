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
  * ``sod_tube``: the Sod tube of the paper's validation (Sect. 4): periodic box x in [-0.5, 1.5),
    left state rho = 1, P = 1 on a close-packed (face-centred cubic) lattice in x < 0.5, right state
    rho = 1/8, P = 0.1 on the same lattice with twice the spacing in x >= 0.5, equal masses, v = 0,
    gamma = 1.4 (u = P / ((gamma-1) rho)).  (On simple cubic lattices the contact sustains a spurious
    pressure jump: the left star density comes out 18% high.)
  * ``advection_step``: the density step of the paper's advection test: rho = 1 for
    0.25 <= x < 0.75 (lattice spacing dx) and 1/8 elsewhere (spacing 2 dx), uniform P, v_x = 1.
  * ``fcc_lattice``: face-centred cubic (close-packed) lattice of n^3 cells x 4 particles in the
    periodic unit box, v = 0, u = 1; the paper's validation runs use close-packed lattices, which,
    unlike the simple cubic one, are stable SPH equilibria.
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


def _block(nx: int, ny: int, x0: float, dx: float) -> list:
    """Cubic lattice of nx x ny x ny points, spacing dx, starting at x0 along x and 0 along y, z."""
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(ny), indexing="ij")
    return [x0 + (ix.reshape(-1) + 0.5) * dx, (iy.reshape(-1) + 0.5) * dx, (iz.reshape(-1) + 0.5) * dx]


def _fcc_block(ncx: int, ncy: int, x0: float, a: float) -> list:
    """Face-centred cubic lattice of ncx x ncy x ncy cells of side a (4 particles per cell), from x0
    along x and 0 along y, z."""
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]]) + 0.25
    ix, iy, iz = np.meshgrid(np.arange(ncx), np.arange(ncy), np.arange(ncy), indexing="ij")
    cells = np.stack([ix.reshape(-1), iy.reshape(-1), iz.reshape(-1)], axis=1).astype(np.float64)
    pos = ((cells[:, None, :] + base[None, :, :]) * a).reshape(-1, 3)
    return [pos[:, 0] + x0, pos[:, 1].copy(), pos[:, 2].copy()]


def sod_tube(nc: int = 64, ncy: int = 6, gamma: float = 1.4, hfact: float = 1.0) -> dict:
    """Sod shock tube in the periodic box [-0.5, 1.5) x [0, ncy/nc)^2 on close-packed (face-centred
    cubic) lattices: nc x ncy x ncy cells of side 1/nc on the left (2 nc particle planes per unit
    length), cells of twice the side on the right (ncy even); equal masses."""
    a = 1.0 / nc
    left = _fcc_block(nc, ncy, -0.5, a)
    right = _fcc_block(nc // 2, ncy // 2, 0.5, 2 * a)
    out = {k: np.concatenate([p, q]) for k, p, q in zip(("x", "y", "z"), left, right)}
    nl, nr = len(left[0]), len(right[0])
    n = nl + nr
    spacing = a / 4 ** (1.0 / 3.0)
    out["u"] = np.concatenate([np.full(nl, 1.0 / ((gamma - 1.0) * 1.0)), np.full(nr, 0.1 / ((gamma - 1.0) * 0.125))])
    out["h"] = np.concatenate([np.full(nl, hfact * spacing), np.full(nr, 2 * hfact * spacing)])
    for k in ("vx", "vy", "vz"):
        out[k] = np.zeros(n)
    out.update(mass=a ** 3 / 4, n=n, dx=spacing, gamma=gamma, box_lo=(-0.5, 0.0, 0.0),
               box_hi=(1.5, ncy * a, ncy * a))
    return out


def advection_step(nx: int = 32, ny: int = 8, hfact: float = 1.2, vx: float = 1.0) -> dict:
    """Density step advected through the periodic box [0, 1) x [0, ny/nx)^2 (uniform pressure)."""
    dx = 1.0 / nx
    a = _block(nx // 8, ny // 2, 0.0, 2 * dx)          # x in [0, 0.25): rho = 1/8
    b = _block(nx // 2, ny, 0.25, dx)                  # x in [0.25, 0.75): rho = 1
    c = _block(nx // 8, ny // 2, 0.75, 2 * dx)         # x in [0.75, 1): rho = 1/8
    out = {k: np.concatenate([p, q, r]) for k, p, q, r in zip(("x", "y", "z"), a, b, c)}
    na, nb, nc = len(a[0]), len(b[0]), len(c[0])
    n = na + nb + nc
    out["u"] = np.concatenate([np.full(na, 8.0), np.full(nb, 1.0), np.full(nc, 8.0)])   # P = (gamma-1) rho u uniform
    out["h"] = np.concatenate([np.full(na, 2 * hfact * dx), np.full(nb, hfact * dx), np.full(nc, 2 * hfact * dx)])
    out["vx"] = np.full(n, vx)
    out["vy"] = np.zeros(n)
    out["vz"] = np.zeros(n)
    out.update(mass=dx ** 3, n=n, dx=dx, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, ny * dx, ny * dx))
    return out


def fcc_lattice(n_cells: int, hfact: float = 1.2, u0: float = 1.0) -> dict:
    """Close-packed (face-centred cubic) lattice: cell side a = 1/n_cells, 4 particles per cell at
    (0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2) a (+ a/4 to keep them off the box faces)."""
    a = 1.0 / n_cells
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]]) + 0.25
    ix, iy, iz = np.meshgrid(np.arange(n_cells), np.arange(n_cells), np.arange(n_cells), indexing="ij")
    cells = np.stack([ix.reshape(-1), iy.reshape(-1), iz.reshape(-1)], axis=1).astype(np.float64)
    pos = ((cells[:, None, :] + base[None, :, :]) * a).reshape(-1, 3)
    n = len(pos)
    spacing = a / 4 ** (1.0 / 3.0)   # (volume per particle)^(1/3)
    out = {"x": pos[:, 0].copy(), "y": pos[:, 1].copy(), "z": pos[:, 2].copy()}
    for k in ("vx", "vy", "vz"):
        out[k] = np.zeros(n)
    out["u"] = np.full(n, float(u0))
    out["h"] = np.full(n, hfact * spacing)
    out.update(mass=1.0 / n, n=n, dx=spacing)
    return out

