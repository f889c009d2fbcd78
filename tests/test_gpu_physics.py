"""GPU density/h iteration (App. F), forces (Sect. 2.1) and KDK step (App. G) against the oracle, in
FP64 and mixed precision.

Tolerances (derived from the arithmetic):
  * h, FP64: both sides stop Newton at |dh|/h^n <= 1e-6; the remaining error after such a step is of
    order (1e-6)^2, so |h_gpu/h_ref - 1| <= 1e-9.
  * forces, FP64, on the same h and Omega: sums of ~60 terms in a different order, each term at most
    c_s^2/h per unit mass: |da| <= 1e-12 * 64 * c_s^2/h_min (about 1e-10 of max|a| here).
  * mixed precision against FP64 (the mixed path's tolerance): rho relative <= 1e-5, a <= 1e-4 of max|a|.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import require_gpu, to_orig

pytestmark = pytest.mark.gpu


def _solver(params, n):
    from paper_2503_09713_gb300 import sph
    return sph.Solver(params, n)


def _gpu_converge(w, precision=0, **kw):
    require_gpu()
    from paper_2503_09713_gb300 import sph
    p = sph.default_params(precision=precision, **kw)
    s = sph.DeviceState.from_numpy(w)
    solver = _solver(p, len(w["x"]))
    solver.converge(s)
    out = s.to_numpy()
    st = solver.stats()
    solver.close()
    ids = out["id"].astype(np.int64)
    return {k: to_orig(out[k], ids) for k in ("h", "rho", "omega", "ax", "ay", "az", "du", "vsig")}, st


def _workload(kind):
    from paper_2503_09713_gb300 import workloads
    if kind == "lattice":
        return workloads.lattice(15, sigma_v=0.1, jitter=0.2, seed=31)
    if kind == "sedov":
        return workloads.sedov(16)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["lattice", "sedov"])
def test_density_fp64_vs_root_and_algF(kind):
    w = _workload(kind)
    g, st = _gpu_converge(w)
    hroot = O.density_root(w["x"], w["y"], w["z"], 1.2, 3.0 * w["dx"])
    assert np.max(np.abs(g["h"] / hroot - 1.0)) < 1e-9
    P = O.Params()
    h, rho, om, it, outer = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
    assert np.max(np.abs(g["h"] / h - 1.0)) < 1e-9
    assert np.max(np.abs(g["rho"] / rho - 1.0)) < 3e-9
    assert np.max(np.abs(g["omega"] - om)) < 1e-8
    # invariant h (rho_sum/m)^(1/3) = hfact at the GPU's h
    rs, _ = O.density_at(w["x"], w["y"], w["z"], g["h"], w["mass"], 1.2)
    assert np.max(np.abs(g["h"] * np.cbrt(rs / w["mass"]) - 1.2)) < 2e-9


def test_density_lattice_value():
    from paper_2503_09713_gb300 import workloads
    w = workloads.perfect_lattice(12)
    g, st = _gpu_converge(w)
    hroot = O.density_root(w["x"], w["y"], w["z"], 1.2, 2.0 * w["dx"])
    assert np.max(np.abs(g["h"] / hroot - 1.0)) < 1e-9
    assert abs(g["h"][0] / w["dx"] - 1.2) < 1e-3
    assert np.max(np.abs(np.stack([g["ax"], g["ay"], g["az"]]))) < 1e-9


def test_cache_stale_and_restart():
    """Start at half the converged h: h must leave chi h^n; the density call reports it and the
    restart (rebuild the cache around the new h) converges to the root."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(12, sigma_v=0.0, jitter=0.1, seed=4)
    w["h"] = 0.5 * w["h"]
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(sph.default_params(), w["n"])
    solver.build_tree(s)
    solver.find_neighbours(s)
    with pytest.raises(sph.SPHError) as e:
        solver.compute_density_h(s)
    assert e.value.code == sph.SPH_ERR_CACHE_STALE
    solver.converge(s)
    out = s.to_numpy()
    solver.close()
    h = to_orig(out["h"], out["id"].astype(np.int64))
    hroot = O.density_root(w["x"], w["y"], w["z"], 1.2, 3.0 * w["dx"])
    assert np.max(np.abs(h / hroot - 1.0)) < 1e-9


def _gpu_forces_given(w, h, om, precision=0, **kw):
    """GPU forces on the oracle's h and Omega (cache built at that h)."""
    require_gpu()
    from paper_2503_09713_gb300 import sph
    d = dict(w)
    d["h"] = h
    d["omega"] = om
    d["rho"] = w["mass"] * (1.2 / h) ** 3
    s = sph.DeviceState.from_numpy(d)
    solver = sph.Solver(sph.default_params(precision=precision, **kw), len(h))
    solver.build_tree(s)
    solver.find_neighbours(s)
    solver.compute_forces(s)
    out = s.to_numpy()
    solver.close()
    ids = out["id"].astype(np.int64)
    return {k: to_orig(out[k], ids) for k in ("ax", "ay", "az", "du", "vsig")}


@pytest.mark.parametrize("kind", ["lattice", "sedov"])
@pytest.mark.parametrize("alpha_u", [1.0, 0.0])
def test_forces_fp64_vs_oracle(kind, alpha_u):
    w = _workload(kind)
    P = O.Params(alpha_u=alpha_u)
    h, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
    ref = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P)
    g = _gpu_forces_given(w, h, om, alpha_u=alpha_u)
    cs2 = (5.0 / 3.0) * (2.0 / 3.0) * np.max(w["u"])
    tol = 1e-12 * 64 * cs2 / np.min(h)
    for k, r in zip(("ax", "ay", "az", "du"), ref[:4]):
        assert np.max(np.abs(g[k] - r)) < tol, k
    assert np.max(np.abs(g["vsig"] / ref[4] - 1)) < 1e-12
    m = w["mass"]
    for k in ("ax", "ay", "az"):
        assert abs(np.sum(m * g[k])) < 1e-12 * np.sum(m * np.abs(g[k])) + 1e-300


@pytest.mark.parametrize("kind", ["lattice", "sedov"])
def test_mixed_vs_fp64(kind):
    w = _workload(kind)
    g64, _ = _gpu_converge(w, precision=0)
    g32, _ = _gpu_converge(w, precision=1)
    assert np.max(np.abs(g32["rho"] / g64["rho"] - 1.0)) < 1e-5
    assert np.max(np.abs(g32["h"] / g64["h"] - 1.0)) < 1e-5
    amax = np.max(np.abs(np.stack([g64["ax"], g64["ay"], g64["az"]])))
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g32[k] - g64[k])) < 1e-4 * amax, k
    dumax = np.max(np.abs(g64["du"]))
    assert np.max(np.abs(g32["du"] - g64["du"])) < 1e-4 * dumax


@pytest.mark.parametrize("precision", [0, 1])
def test_step_vs_oracle(precision):
    """One KDK step from the same converged state with the same dt (taken from the oracle)."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(16, sigma_v=0.1, jitter=0.1, seed=77)
    P = O.Params()
    h, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
    ax, ay, az, du, vs = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P)
    dt = O.cfl(h, vs, ax, ay, az, P)
    ref = {k: w[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    ref.update({k: v.copy() for k, v in (("h", h), ("ax", ax), ("ay", ay), ("az", az), ("du", du), ("rho", rho),
                                          ("omega", om), ("vsig", vs))})
    dtn_ref, it, dvr = O.step(ref, w["mass"], P, dt)     # in place on ref; h, a, ... keep the step-n values

    d = dict(w)
    d.update(h=h, rho=rho, omega=om, ax=ax, ay=ay, az=az, du=du, vsig=vs)
    s = sph.DeviceState.from_numpy(d)
    solver = sph.Solver(sph.default_params(precision=precision), w["n"])
    used, dtn = solver.step(s, dt)
    dvr_gpu = solver.stats()["dv_ratio"]
    out = s.to_numpy()
    solver.close()
    ids = out["id"].astype(np.int64)
    g = {k: to_orig(out[k], ids) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du")}
    assert used == dt
    tol_h = 1e-9 if precision == 0 else 1e-5
    assert np.max(np.abs(g["h"] / ref["h"] - 1)) < tol_h
    amax = np.max(np.abs(np.stack([ref["ax"], ref["ay"], ref["az"]])))
    tol_a = 1e-8 * amax if precision == 0 else 1e-4 * amax
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - ref[k])) < tol_a, k
    for k in ("x", "y", "z"):
        dxk = np.abs(g[k] - ref[k])
        dxk = np.minimum(dxk, 1.0 - dxk)
        assert np.max(dxk) < 1e-14
    assert abs(dtn / dtn_ref - 1) < (1e-8 if precision == 0 else 1e-4)
    if precision == 0:   # step-quality ratio max|dv| / rms|v| (its |dv| and |v|^2 are FP32 statistics)
        assert dvr > 0 and abs(dvr_gpu / dvr - 1) < 1e-5


KERNEL_HFACT = [("M4", 0, 1.2), ("M5", 1, 1.2), ("M6", 2, 1.0), ("C2", 3, 1.2), ("C4", 4, 1.2), ("C6", 5, 1.2)]


@pytest.mark.parametrize("name,kernel,hfact", KERNEL_HFACT)
@pytest.mark.parametrize("precision", [0, 1])
def test_kernel_family_vs_oracle(name, kernel, hfact, precision):
    """Every kernel of Sect. 2.1 through the GPU path (cache radius R chi h, density root, forces)
    against the oracle with the same kernel: converged h, rho and accelerations."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(14, sigma_v=0.1, jitter=0.1, seed=60 + kernel, hfact=hfact)
    w["u"] = 1.0 + 0.5 * np.random.default_rng(kernel).uniform(size=w["n"])
    P = O.Params(kernel=kernel, hfact=hfact)
    h, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
    ax, ay, az, du, vs = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P)
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(sph.default_params(precision=precision, kernel=kernel, hfact=hfact), w["n"])
    solver.converge(s)
    out = s.to_numpy()
    solver.close()
    ids = out["id"].astype(np.int64)
    g = {k: to_orig(out[k], ids) for k in ("h", "rho", "ax", "ay", "az", "du")}
    amax = np.max(np.abs(np.stack([ax, ay, az])))
    tol_h, tol_a = (1e-9, 1e-8) if precision == 0 else (1e-5, 1e-4)
    assert np.max(np.abs(g["h"] / h - 1)) < tol_h
    assert np.max(np.abs(g["rho"] / rho - 1)) < 3 * tol_h
    for k, ref in (("ax", ax), ("ay", ay), ("az", az)):
        assert np.max(np.abs(g[k] - ref)) < tol_a * amax, k
