"""Shock switch, per-particle viscosity, corrector re-runs and the CFL multiplier (App. G) through
the GPU step against the oracle's step with the same settings."""
import numpy as np
import pytest

import oracle as O
from gpu_common import require_gpu, to_orig

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig", "alpha")


def _converged(w, P):
    h, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
    alpha = w.get("alpha")
    if alpha is None:
        ax, ay, az, du, vs = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P)
    else:
        ax, ay, az, du, vs = O.forces_alpha(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, alpha,
                                            w["mass"], P)
    st = {k: w[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    st.update(h=h, rho=rho, omega=om, ax=ax, ay=ay, az=az, du=du, vsig=vs)
    if alpha is not None:
        st["alpha"] = alpha.copy()
    return st


def _gpu_steps(start, mass, params, dts, n):
    from paper_2503_09713_gb300 import sph
    d = dict(start)
    d["mass"] = mass
    s = sph.DeviceState.from_numpy(d)
    solver = sph.Solver(params, n)
    info = []
    for dt in dts:
        used, dtn = solver.step(s, dt)
        st = solver.stats()
        info.append((used, dtn, st["corrector_passes"], st["cfl_multiplier"]))
    out = s.to_numpy()
    solver.close()
    ids = out["id"].astype(np.int64)
    return {k: to_orig(out[k], ids) for k in FIELDS if k in out}, info


def _compare(g, ref, precision, what):
    amax = np.max(np.abs(np.stack([ref["ax"], ref["ay"], ref["az"]])))
    tol_h, tol_a = (1e-9, 1e-8) if precision == 0 else (1e-5, 1e-4)
    assert np.max(np.abs(g["h"] / ref["h"] - 1)) < tol_h, what
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - ref[k])) < tol_a * amax, what + " " + k
    vmax = np.max(np.abs(np.stack([ref["vx"], ref["vy"], ref["vz"]]))) + 1e-300
    for k in ("vx", "vy", "vz"):
        assert np.max(np.abs(g[k] - ref[k])) < (1e-10 if precision == 0 else 1e-4) * vmax, what + " " + k


@pytest.mark.parametrize("precision", [0, 1])
def test_switch_step_vs_oracle(precision):
    """Two steps with av_switch = 1 from a converged state with a random alpha field: alpha, h, a
    and v against the oracle's step (FP64: alpha to 1e-9; mixed: FP32 gradient sums, 1e-3)."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(14, sigma_v=0.3, jitter=0.1, seed=71)
    rng = np.random.default_rng(5)
    w["u"] = 1.0 + 0.5 * rng.uniform(size=w["n"])
    w["vx"] = w["vx"] - 0.4 * np.sin(2 * np.pi * w["x"])   # a converging region
    w["alpha"] = rng.uniform(0.1, 0.9, size=w["n"])
    P = O.Params(av_switch=1)
    start = _converged(w, P)
    dt = 0.5 * O.cfl(start["h"], start["vsig"], start["ax"], start["ay"], start["az"], P)
    ref = {k: v.copy() for k, v in start.items()}
    for _ in range(2):
        O.step(ref, w["mass"], P, dt)
    g, _ = _gpu_steps(start, w["mass"], sph.default_params(precision=precision, av_switch=1), [dt, dt], w["n"])
    assert np.any(np.abs(ref["alpha"] - start["alpha"]) > 1e-3)   # the switch acted
    assert np.max(np.abs(g["alpha"] - ref["alpha"])) < (1e-9 if precision == 0 else 1e-3)
    _compare(g, ref, precision, "switch")


def test_corrector_reruns_and_multiplier_vs_oracle():
    """Sedov start with eps_v = 1e-2: the corrector passes, the CFL multiplier, the next time
    step and the state after three steps against the oracle (FP64)."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.sedov(12, seed=77)
    P = O.Params(eps_v=1e-2, max_corr=3, lambda_stiff=1.0)
    start = _converged(w, P)
    dt0 = O.cfl(start["h"], start["vsig"], start["ax"], start["ay"], start["az"], P)
    ref = {k: v.copy() for k, v in start.items()}
    dts, passes, lams = [], [], []
    dt = dt0
    for _ in range(3):
        dts.append(dt)
        dt, _, _ = O.step(ref, w["mass"], P, dt)
        passes.append(ref["corrector_passes"])
        lams.append(ref["lambda_cfl"])
    assert max(passes) >= 2   # the re-runs were exercised
    g, info = _gpu_steps(start, w["mass"], sph.default_params(eps_v=1e-2, max_corr=3, lambda_stiff=1.0), dts,
                         w["n"])
    assert [i[2] for i in info] == passes
    assert [i[3] for i in info] == pytest.approx(lams, rel=1e-14)
    assert info[-1][1] == pytest.approx(dt, rel=1e-8)
    _compare(g, ref, 0, "re-runs")
