"""The batched ensemble at full size and split over ranks.

* The 256-box ensemble workload of the benchmark (14.0 M particles, boxes of 13^3 .. 64^3, the box
  index in the top 8 bits of the keys and 18 Morton bits per axis) in mixed precision and in FP64:
  converged state and one step with a common time step, compared box by box with the oracle (the
  equations of Sect. 2.1 and the iteration of App. F per box) on 8 boxes: the largest, the smallest,
  both adiabatic indices and random others.  The oracle's step starts from the GPU's converged state
  of that box, so both sides advance the same input.
* A context holding half of a small ensemble (the boxes one of two ranks gets) gives, box by box,
  the same bits as the context holding all of it: boxes are independent, so sharding them over GPUs
  changes no result.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import require_gpu, to_orig

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig")


def _pick(boxes, k=8, seed=5):
    n = np.array([b["n"] for b in boxes])
    g = np.array([b["gamma"] for b in boxes])
    sel = {int(np.argmax(n)), int(np.argmin(n)), int(np.flatnonzero(g > 1.5)[0]), int(np.flatnonzero(g < 1.5)[0])}
    rng = np.random.default_rng(seed)
    while len(sel) < k:
        sel.add(int(rng.integers(0, len(boxes))))
    return sorted(sel)


def _compare(g, ref, lo, hi, precision, what):
    amax = np.max(np.abs(np.stack([ref["ax"], ref["ay"], ref["az"]])))
    tol_h, tol_a = (1e-9, 1e-8 * amax) if precision == 0 else (1e-5, 1e-4 * amax)
    assert np.max(np.abs(g["h"][lo:hi] / ref["h"] - 1)) < tol_h, what
    assert np.max(np.abs(g["rho"][lo:hi] / ref["rho"] - 1)) < tol_h, what
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k][lo:hi] - ref[k])) < tol_a, what + " " + k
    for k in ("x", "y", "z"):
        d = np.abs(g[k][lo:hi] - ref[k])
        assert np.max(np.minimum(d, 1 - d)) < 1e-13, what + " " + k


@pytest.mark.parametrize("precision", [1, 0])
def test_full_ensemble_against_oracle(precision):
    torch = require_gpu()
    from paper_2503_09713_gb300 import replicas, sph, workloads
    boxes = workloads.ensemble(256, seed=12349)
    part = replicas.ensemble_shard(boxes, 1, 0)
    off = part["offsets"]
    assert min(b["n"] for b in boxes) == 2197 and max(b["n"] for b in boxes) == 262144
    sel = _pick(boxes)
    refs = {}
    for b in sel:
        P = O.Params(gamma=boxes[b]["gamma"])
        w = boxes[b]
        h, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
        ax, ay, az, du, vs = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P)
        st = {k: w[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
        st.update(h=h, rho=rho, omega=om, ax=ax, ay=ay, az=az, du=du, vsig=vs)
        refs[b] = (st, P)
    s = sph.DeviceState.from_numpy(part["state"])
    solver = sph.Solver.batch(sph.default_params(precision=precision), off, part["mass"], part["gamma"])
    solver.converge(s)
    out = s.to_numpy()
    g0 = {k: to_orig(out[k], out["id"].astype(np.int64)) for k in FIELDS}
    for b in sel:
        _compare(g0, refs[b][0], off[b], off[b + 1], precision, f"box {b} (n={boxes[b]['n']}) converged")
    # one step of every box with the smallest CFL step of the ensemble
    dt = float(np.min(solver.batch_dt()))
    used, _ = solver.step(s, dt)
    assert used == dt
    out1 = s.to_numpy()
    g1 = {k: to_orig(out1[k], out1["id"].astype(np.int64)) for k in FIELDS}
    for b in sel:
        lo, hi = off[b], off[b + 1]
        st = {k: g0[k][lo:hi].copy() for k in FIELDS}     # the GPU's converged state of this box
        O.step(st, boxes[b]["mass"], refs[b][1], dt)
        _compare(g1, st, lo, hi, precision, f"box {b} after one step")
    solver.close()
    del s
    torch.cuda.empty_cache()


def test_half_ensemble_context_equals_full_context():
    require_gpu()
    from paper_2503_09713_gb300 import replicas, sph, workloads
    boxes = workloads.ensemble(8, seed=777, n_max=30000)
    full = replicas.ensemble_shard(boxes, 1, 0)
    half = replicas.ensemble_shard(boxes, 2, 1)
    assert 0 < len(half["boxes"]) < 8
    res = {}
    for name, part in (("full", full), ("half", half)):
        s = sph.DeviceState.from_numpy(part["state"])
        solver = sph.Solver.batch(sph.default_params(precision=sph.SPH_MIXED), part["offsets"], part["mass"],
                                  part["gamma"])
        solver.converge(s)
        for _ in range(2):
            solver.step(s, 0.0)          # every box by its own CFL step
        out = s.to_numpy()
        res[name] = ({k: to_orig(out[k], out["id"].astype(np.int64)) for k in FIELDS}, part)
        solver.close()
    gf, pf = res["full"]
    gh, ph = res["half"]
    for k, b in enumerate(ph["boxes"]):
        lo_h, hi_h = ph["offsets"][k], ph["offsets"][k + 1]
        lo_f, hi_f = pf["offsets"][b], pf["offsets"][b + 1]
        for f in FIELDS:
            assert np.array_equal(gh[f][lo_h:hi_h], gf[f][lo_f:hi_f]), (b, f)
