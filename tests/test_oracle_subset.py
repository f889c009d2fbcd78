"""Pins of the oracle's sampled evaluation (orc_subset_forces, orc_subset_neighbours) and of its CFL
time step (orc_cfl, App. G "Choice of the timestep").

The sampled functions are the only check of the largest GPU parity tests (256^3 and 512^3), so they
are pinned here against the oracle's full evaluation -- neighbour lists of every particle, the root
of the density equation for every particle, Omega from Eq. sphomega and the pair forces of Eqs.
sphvel / sphuint -- on small periodic boxes, element by element.  Both a uniform lattice and a
Sedov-like box (compressed centre, so h varies by a factor ~1.6, hot centre, radial outflow) are
used, and the sampled particles include those on the faces and in a corner of the box, where the
nearest periodic image matters.  The CFL step is pinned by closed forms.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_09713_gb300 import workloads as WL


def _uniform(n_side=12, seed=21):
    w = WL.lattice(n_side, sigma_v=0.1, seed=seed)
    rng = np.random.default_rng(seed + 1)
    w["u"] = 1.0 + 0.3 * rng.uniform(-1, 1, size=w["n"])   # pressure differences: conductivity at work
    return w


def _sedov_like(n_side=12, seed=22):
    """Lattice compressed towards the centre (r -> r (0.4 + 0.6 r / 0.4) inside r < 0.4), u peaked at
    the centre, radial outflow: h varies by a factor ~1.6 over the box."""
    w = WL.lattice(n_side, sigma_v=0.0, seed=seed)
    c = 0.5
    d = np.stack([w["x"] - c, w["y"] - c, w["z"] - c])
    r = np.sqrt((d * d).sum(0))
    f = np.where(r < 0.4, 0.4 + 0.6 * r / 0.4, 1.0)
    p = c + d * f
    w["x"], w["y"], w["z"] = p[0], p[1], p[2]
    w["u"] = 1e-3 + 5.0 * np.exp(-(r / 0.15) ** 2)
    rr = np.maximum(r, 1e-12)
    vr = 0.5 * np.exp(-(r / 0.2) ** 2)
    w["vx"], w["vy"], w["vz"] = vr * d[0] / rr, vr * d[1] / rr, vr * d[2] / rr
    return w


def _sample(w, seed):
    """Random particles plus the ones nearest to each face of the box and to one corner."""
    rng = np.random.default_rng(seed)
    idx = list(rng.choice(w["n"], 12, replace=False))
    for k in ("x", "y", "z"):
        idx.append(int(np.argmin(w[k])))
        idx.append(int(np.argmax(w[k])))
    corner = (np.minimum(w["x"], 1 - w["x"]) + np.minimum(w["y"], 1 - w["y"]) + np.minimum(w["z"], 1 - w["z"]))
    idx.append(int(np.argmin(corner)))
    return np.array(sorted(set(idx)), dtype=np.int64)


@pytest.mark.parametrize("make", [_uniform, _sedov_like])
def test_subset_forces_equals_full_oracle(make):
    w = make()
    P = O.Params()
    h_hi = 2.0 * w["dx"]
    args = [w[k] for k in ("x", "y", "z")]
    h = O.density_root(*args, P.hfact, h_hi, method=0)
    assert np.all(np.isfinite(h))
    if make is _sedov_like:
        assert h.max() / h.min() > 1.4          # the h field does vary
    _, om = O.density_at(*args, h, w["mass"], P.hfact, method=0)
    ax, ay, az, du, vs = O.forces(*args, w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P, method=0)
    idx = _sample(w, 5)
    r = O.subset_forces(*args, w["vx"], w["vy"], w["vz"], w["u"], w["mass"], P, idx, h_hi)
    assert np.max(np.abs(r["h"] / h[idx] - 1)) < 1e-12
    assert np.max(np.abs(r["omega"] - om[idx])) < 1e-12
    amax = np.max(np.abs(np.stack([ax, ay, az])))
    for k, full in (("ax", ax), ("ay", ay), ("az", az)):
        assert np.max(np.abs(r[k] - full[idx])) < 1e-12 * amax, k
    assert np.max(np.abs(r["du"] - du[idx])) < 1e-12 * np.max(np.abs(du))
    assert np.max(np.abs(r["vsig"] / vs[idx] - 1)) < 1e-12


@pytest.mark.parametrize("make", [_uniform, _sedov_like])
def test_subset_neighbours_equals_full_oracle(make):
    w = make()
    rng = np.random.default_rng(8)
    hc = w["dx"] * rng.uniform(0.9, 1.6, size=w["n"])   # unequal h: the max(h_a, h_b) criterion matters
    s = 2.0 * 1.1
    args = [w[k] for k in ("x", "y", "z")]
    off, ids = O.neighbours(*args, hc, s, method=0)
    idx = _sample(w, 9)
    so, si = O.subset_neighbours(*args, hc, s, idx)
    assert len(so) == len(idx) + 1
    for k, a in enumerate(idx):
        assert np.array_equal(np.sort(si[so[k]:so[k + 1]]), np.sort(ids[off[a]:off[a + 1]])), a


def test_cfl_closed_forms():
    """dt = min_a min(C_cour h_a / v_sig,a, C_force sqrt(h_a / |a_a|)) with distinct C_cour, C_force,
    so that a swap of the two factors, of h and v_sig, or a dropped square root changes the result."""
    P = O.Params(c_cour=0.3, c_force=0.25)
    z = np.zeros(2)
    # no acceleration: the signal-speed term alone, smallest over particles
    assert O.cfl(np.array([0.1, 0.2]), np.array([2.0, 1.0]), z, z, z, P) == pytest.approx(0.3 * 0.05, rel=1e-15)
    # the force term wins: |a| = 5, h = 0.01 -> 0.25 sqrt(0.002); the Courant term 0.3 * 0.01 / 1e-3 = 3
    dt = O.cfl(np.array([0.01]), np.array([1e-3]), np.array([3.0]), np.array([4.0]), np.array([0.0]), P)
    assert dt == pytest.approx(0.25 * math.sqrt(0.01 / 5.0), rel=1e-15)
    # mixed: particle 0 limited by its signal speed, particle 1 by its acceleration
    h = np.array([0.02, 0.04])
    vs = np.array([1.0, 0.01])
    ax = np.array([0.0, 100.0])
    dt = O.cfl(h, vs, ax, z, z, P)
    assert dt == pytest.approx(min(0.3 * 0.02 / 1.0, 0.25 * math.sqrt(0.04 / 100.0)), rel=1e-15)


def test_cfl_of_lattice_at_rest():
    """Perfect lattice at rest with uniform u: no pair approaches, so v_sig = alpha_AV c_s, and the
    pressure forces cancel (|a| at rounding level), so dt = C_cour h / (alpha_AV sqrt(gamma (gamma-1) u))."""
    s = WL.perfect_lattice(10)
    P = O.Params()
    h, rho, om, _, _ = O.density_algF(s["x"], s["y"], s["z"], s["h"], s["mass"], P)
    ax, ay, az, du, vs = O.forces(s["x"], s["y"], s["z"], s["vx"], s["vy"], s["vz"], s["u"], h, om, s["mass"], P)
    cs = math.sqrt(P.gamma * (P.gamma - 1.0) * 1.0)
    assert np.allclose(vs, P.alpha_av * cs, rtol=1e-14, atol=0)
    dt = O.cfl(h, vs, ax, ay, az, P)
    assert dt == pytest.approx(P.c_cour * h.min() / (P.alpha_av * cs), rel=1e-12)
