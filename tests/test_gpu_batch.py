"""Batched ensemble (sph_batch_create): several independent periodic boxes of different sizes,
masses and adiabatic indices in one context, against the oracle run box by box."""
import numpy as np
import pytest

import oracle as O
from gpu_common import require_gpu, to_orig

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig")


def _ensemble():
    from paper_2503_09713_gb300 import workloads
    sides = [10, 12, 9, 13, 16, 11]
    sigmas = [0.05, 0.2, 0.1, 0.02, 0.3, 0.15]
    gammas = [5 / 3, 7 / 5, 5 / 3, 7 / 5, 5 / 3, 7 / 5]
    boxes = [workloads.lattice(s, sigma_v=sg, jitter=0.1, seed=200 + i) for i, (s, sg) in enumerate(zip(sides, sigmas))]
    off = np.concatenate([[0], np.cumsum([b["n"] for b in boxes])]).astype(np.int64)
    cat = {k: np.concatenate([b[k] for b in boxes]) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h")}
    cat["mass"] = 1.0
    return boxes, off, np.array([b["mass"] for b in boxes]), np.array(gammas), cat


def _oracle_box(b, gamma):
    P = O.Params(gamma=gamma)
    h, rho, om, _, _ = O.density_algF(b["x"], b["y"], b["z"], b["h"], b["mass"], P)
    ax, ay, az, du, vs = O.forces(b["x"], b["y"], b["z"], b["vx"], b["vy"], b["vz"], b["u"], h, om, b["mass"], P)
    st = {k: b[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    st.update(h=h, rho=rho, omega=om, ax=ax, ay=ay, az=az, du=du, vsig=vs)
    return st, P


def _check(g, ref, lo, hi, precision, what):
    amax = np.max(np.abs(np.stack([ref["ax"], ref["ay"], ref["az"]])))
    tol_h, tol_a = (1e-9, 1e-8 * amax) if precision == 0 else (1e-5, 1e-4 * amax)
    assert np.max(np.abs(g["h"][lo:hi] / ref["h"] - 1)) < tol_h, what
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k][lo:hi] - ref[k])) < tol_a, what + " " + k
    for k in ("x", "y", "z"):
        d = np.abs(g[k][lo:hi] - ref[k])
        assert np.max(np.minimum(d, 1 - d)) < 1e-13, what + " " + k


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_oracle_box_by_box(precision):
    require_gpu()
    from paper_2503_09713_gb300 import sph
    boxes, off, mass, gam, cat = _ensemble()
    refs = [_oracle_box(b, g) for b, g in zip(boxes, gam)]
    s = sph.DeviceState.from_numpy(cat)
    solver = sph.Solver.batch(sph.default_params(precision=precision), off, mass, gam)
    solver.converge(s)
    out = s.to_numpy()
    ids = out["id"].astype(np.int64)
    assert all(np.all((ids[off[b]:off[b + 1]] >= off[b]) & (ids[off[b]:off[b + 1]] < off[b + 1]))
               for b in range(len(boxes)))                     # particles stay in their box
    g0 = {k: to_orig(out[k], ids) for k in FIELDS}
    gs = solver.export_tree()["group_start"]                   # groups: runs of <= 32 inside one box
    assert gs[0] == 0 and gs[-1] == off[-1] and np.all(np.diff(gs) >= 1) and np.all(np.diff(gs) <= 32)
    box = np.searchsorted(off, np.arange(off[-1]), side="right") - 1
    assert np.array_equal(box[gs[:-1]], box[gs[1:] - 1])
    dts = solver.batch_dt()
    for b, (ref, P) in enumerate(refs):
        _check(g0, ref, off[b], off[b + 1], precision, f"box {b} converged")
        dt_ref = O.cfl(ref["h"], ref["vsig"], ref["ax"], ref["ay"], ref["az"], P)
        assert abs(dts[b] / dt_ref - 1) < (1e-8 if precision == 0 else 1e-4)
    solver.close()

    # one step of every box with a common dt, from the oracle's converged states
    dt = min(O.cfl(r["h"], r["vsig"], r["ax"], r["ay"], r["az"], P) for r, P in refs)
    start = {k: np.concatenate([r[k] for r, _ in refs]) for k in FIELDS}
    start["mass"] = 1.0
    s1 = sph.DeviceState.from_numpy(start)
    solver1 = sph.Solver.batch(sph.default_params(precision=precision), off, mass, gam)
    used, _ = solver1.step(s1, dt)
    assert used == dt
    out1 = s1.to_numpy()
    g1 = {k: to_orig(out1[k], out1["id"].astype(np.int64)) for k in FIELDS}
    for b, (ref, P) in enumerate(refs):
        r1 = {k: v.copy() for k, v in ref.items()}
        O.step(r1, boxes[b]["mass"], P, dt)
        _check(g1, r1, off[b], off[b + 1], precision, f"box {b} after one step")
    # a second step with each box's own CFL step
    used2, _ = solver1.step(s1, 0.0)
    assert used2 > 0
    solver1.close()
