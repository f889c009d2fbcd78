"""Validation runs of the GPU path against closed forms (the paper's Sect. 4 tests): advection of a
density step over many box crossings, the Sod tube against the exact Riemann solution, and the
Sedov-Taylor blast radius and energy conservation."""
import numpy as np
import pytest

from exact_solutions import riemann_sample, sedov_radius
from gpu_common import require_gpu, to_orig

pytestmark = pytest.mark.gpu


def _run(w, params, t_end, max_steps=20000):
    """Converge, then CFL steps until t_end (the last step shortened to land on it)."""
    from paper_2503_09713_gb300 import sph
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(params, w["n"])
    solver.converge(s)
    t, steps, dt = 0.0, 0, solver.stats()["dt_next"]
    while t < t_end * (1 - 1e-12) and steps < max_steps:
        used, dt = solver.step(s, min(dt, t_end - t))
        t += used
        steps += 1
    out = s.to_numpy()
    solver.close()
    ids = out["id"].astype(np.int64)
    return {k: to_orig(out[k], ids) for k in out if k not in ("id", "mass")}, t, steps


def _energy(st, m):
    return float(np.sum(m * (st["u"] + 0.5 * (st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2))))


def _advect(w, p, steps, dt):
    from paper_2503_09713_gb300 import sph
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(p, w["n"])
    solver.converge(s)
    for _ in range(steps):
        solver.step(s, dt)
    out = s.to_numpy()
    solver.close()
    ids = out["id"].astype(np.int64)
    return {k: to_orig(out[k], ids) for k in ("x", "y", "z", "rho", "vx", "vy", "u")}


def _periodic_diff(a, b, L):
    d = np.abs(a - b)
    return np.minimum(d, L - d)


def test_advection_over_box_crossings():
    """The paper's advection test (11 box crossings) on a lattice in equilibrium: the signal speed of
    uniform motion is c_s whatever the velocity, so v = (110, 50, 30) with dt = 0.01 makes 11, 5
    and 3 crossings in 10 steps, as v_x = 1 does along x at t = 11; every particle is back at its
    initial position modulo the box to rounding, with the initial density (the periodic wrap of the
    predictor, the tree and the cache leave no trace)."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.perfect_lattice(16)
    w["vx"], w["vy"], w["vz"] = np.full(w["n"], 110.0), np.full(w["n"], 50.0), np.full(w["n"], 30.0)
    g = _advect(w, sph.default_params(), 10, 0.01)
    for k in ("x", "y", "z"):
        assert np.max(_periodic_diff(g[k], w[k], 1.0)) < 1e-10, k
    assert np.max(np.abs(g["vx"] - 110.0)) < 1e-9
    assert np.ptp(g["rho"]) < 1e-9 * np.mean(g["rho"])


def test_advected_density_step_is_galilean_invariant():
    """A pressure-balanced density step (rho 1 and 1/8 on lattices of spacing dx and 2 dx; its
    contact is not in exact SPH equilibrium) moving at v_x = 1 across the periodic boundary: after
    30 steps the state equals the run at rest shifted by v_x t (positions, density, velocity, u) to
    rounding."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    runs = []
    for vx in (1.0, 0.0):
        w = workloads.advection_step(32, 8, vx=vx)
        runs.append(_advect(w, sph.default_params(box_lo=w["box_lo"], box_hi=w["box_hi"]), 30, 0.01))
    a, b = runs
    assert np.max(_periodic_diff(a["x"], (b["x"] + 0.3) % 1.0, 1.0)) < 1e-10
    for k in ("y", "z"):
        assert np.max(_periodic_diff(a[k], b[k], w["box_hi"][1])) < 1e-10, k
    assert np.max(np.abs(a["rho"] / b["rho"] - 1)) < 1e-10
    assert np.max(np.abs((a["vx"] - 1.0) - b["vx"])) < 1e-10 and np.max(np.abs(a["u"] / b["u"] - 1)) < 1e-10


def _sod_l2(nc, precision):
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.sod_tube(nc, 6)
    w["alpha"] = np.full(w["n"], 1.0)
    p = sph.default_params(precision=precision, kernel=sph.SPH_KERNEL_M6, hfact=1.0, gamma=1.4,
                           box_lo=w["box_lo"], box_hi=w["box_hi"], av_switch=1)
    out, t, steps = _run(w, p, 0.245)
    assert abs(t - 0.245) < 1e-12
    sel = (out["x"] >= 0.0) & (out["x"] < 1.0)
    rho_e, u_e, p_e = riemann_sample(out["x"][sel], t, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    P = 0.4 * out["rho"][sel] * out["u"][sel]
    l2 = {k: float(np.sqrt(np.mean((a - b) ** 2))) for k, a, b in
          (("rho", out["rho"][sel], rho_e), ("v", out["vx"][sel], u_e), ("P", P, p_e))}
    mom = float(np.sum(w["mass"] * out["vx"]))
    return l2, mom, w["mass"] * w["n"]


@pytest.mark.parametrize("precision", [0, 1])
def test_sod_tube_against_exact_solution(precision):
    """Sod tube (M6, hfact 1.0, shock switch, conductivity, gamma 1.4) at t = 0.245 against the exact
    Riemann solution on 0 <= x < 1 (the region the second, periodic interface has not reached):
    L2 errors (the paper's norm over particles) of rho, v_x and P with 128 particle planes per unit
    length on the left (close-packed lattices, as in the paper; measured 0.016, 0.043, 0.014 in both
    precisions, against 0.020, 0.061, 0.021 with 64 planes and 0.013, 0.035, 0.011 with 256), lower
    than with 64 planes (convergence), momentum conserved to rounding."""
    require_gpu()
    l2, mom, mtot = _sod_l2(64, precision)
    assert l2["rho"] < 0.025 and l2["v"] < 0.06 and l2["P"] < 0.02, l2
    assert abs(mom) < (1e-10 if precision == 0 else 1e-5) * mtot, mom
    if precision == 0:
        coarse, _, _ = _sod_l2(32, 0)
        for k in ("rho", "v", "P"):
            assert l2[k] < coarse[k], (k, l2, coarse)


def test_sedov_blast_radius_and_energy():
    """Sedov-Taylor blast (E = 1 in the uniform unit box, gamma 5/3, M6 with hfact 1.0, shock switch,
    CFL 0.1 and the corrector check eps_v = 1e-2 as in the paper's test): the radius of the radial
    density maximum follows R = xi_0 (E t^2/rho)^(1/5) within the smoothing scale at t = 0.02 and
    0.05, and the total energy is conserved to 1e-4 (measured 6e-5; 3e-4 without the check)."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.sedov(40, seed=12346, hfact=1.0)
    w["alpha"] = np.full(w["n"], 1.0)
    p = sph.default_params(kernel=sph.SPH_KERNEL_M6, hfact=1.0, av_switch=1, c_cour=0.1, c_force=0.1,
                           eps_v=1e-2)
    e0 = _energy(w, w["mass"])
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(p, w["n"])
    solver.converge(s)
    t, dt = 0.0, solver.stats()["dt_next"]
    for t_end in (0.02, 0.05):
        while t < t_end * (1 - 1e-12):
            used, dt = solver.step(s, min(dt, t_end - t))
            t += used
        out = s.to_numpy()
        r = np.sqrt((out["x"] - 0.5) ** 2 + (out["y"] - 0.5) ** 2 + (out["z"] - 0.5) ** 2)
        edges = np.linspace(0.0, 0.48, 49)
        k = np.digitize(r, edges) - 1
        prof = np.array([out["rho"][k == i].mean() if np.any(k == i) else 0.0 for i in range(48)])
        i = int(np.argmax(prof))
        r_peak = 0.5 * (edges[i] + edges[i + 1])
        R = sedov_radius(t)
        assert abs(r_peak - R) < 3.0 * w["dx"], (t, r_peak, R)
        assert prof[i] > 1.5, prof[i]   # a strong shock (the exact jump is 4, smoothed over 2 h)
        assert abs(_energy(out, w["mass"]) / e0 - 1) < 1e-4
    solver.close()


def _bump(q):
    """Cubic B-spline bump of radius 2 (unnormalised), used only to spread the blast energy."""
    w = np.zeros_like(q)
    a, b = q < 1.0, (q >= 1.0) & (q < 2.0)
    w[a] = 1.0 - 1.5 * q[a] ** 2 + 0.75 * q[a] ** 3
    w[b] = 0.25 * (2.0 - q[b]) ** 3
    return w


def _sedov_box12(n_side):
    """The paper's Sedov-Taylor set-up (Sect. 4.4): rho = 1, u ~ 0, gamma 5/3 in the box [-0.6, 0.6]^3,
    E = 1 spread over the particles within 2 h0 of the centre (sum m u = 1), here on a cubic lattice."""
    from paper_2503_09713_gb300 import workloads
    side = 1.2
    w = workloads.lattice(n_side, sigma_v=0.0, u0=1e-8, hfact=1.0, seed=12346)
    for k in ("x", "y", "z"):
        w[k] = (w[k] - 0.5) * side
    w["h"] = w["h"] * side
    w["mass"] = side ** 3 / w["n"]
    r = np.sqrt(w["x"] ** 2 + w["y"] ** 2 + w["z"] ** 2)
    bw = _bump(r / w["h"][0])
    w["u"] = w["u"] + bw / (w["mass"] * bw.sum())
    w["alpha"] = np.full(w["n"], 1.0)
    return w


def test_sedov_profiles_approach_similarity_solution():
    """The Sedov-Taylor comparison of the paper's Sect. 4.4: M6 with hfact 1.0, shock switch, CFL 0.1,
    corrector check 1e-2, box [-0.6, 0.6]^3, t = 0.1 (R = 0.458), and the paper's norm (RMS over all
    particles) of rho, v_r and P against the exact similarity solution, at 32^3, 64^3 and 96^3.
    These sizes lie below the paper's (26^3 .. 840^3): the post-shock density structure (width ~0.05 R)
    is not resolved yet, so the errors fall slowly; the test requires the errors (L2 and mean absolute)
    at 64^3 and 96^3 to lie below those at 32^3 and the 96^3 ones below the 64^3 ones, the density
    peak to sit within 2 particle spacings of R, and energy to be conserved to 1e-4."""
    require_gpu()
    from exact_solutions import sedov_profile
    from paper_2503_09713_gb300 import sph
    g, t_end = 5.0 / 3.0, 0.1
    l1, l2 = [], []
    for n_side in (32, 64, 96):
        w = _sedov_box12(n_side)
        p = sph.default_params(kernel=sph.SPH_KERNEL_M6, hfact=1.0, av_switch=1, c_cour=0.1, c_force=0.1,
                               eps_v=1e-2, box_lo=(-0.6, -0.6, -0.6), box_hi=(0.6, 0.6, 0.6))
        e0 = _energy(w, w["mass"])
        s = sph.DeviceState.from_numpy(w)
        solver = sph.Solver(p, w["n"])
        solver.converge(s)
        t, dt = 0.0, solver.stats()["dt_next"]
        while t < t_end * (1 - 1e-12):
            used, dt = solver.step(s, min(dt, t_end - t))
            t += used
        out = s.to_numpy()
        solver.close()
        assert abs(_energy(out, w["mass"]) / e0 - 1) < 1e-4
        d = np.stack([out["x"], out["y"], out["z"]])
        r = np.sqrt((d * d).sum(0))
        v_r = (out["vx"] * d[0] + out["vy"] * d[1] + out["vz"] * d[2]) / np.maximum(r, 1e-12)
        P = (g - 1.0) * out["rho"] * out["u"]
        rho_e, v_e, P_e = sedov_profile(r, t, g)
        pairs = ((out["rho"], rho_e), (v_r, v_e), (P, P_e))
        l2.append([float(np.sqrt(np.mean((a - b) ** 2))) for a, b in pairs])
        l1.append([float(np.mean(np.abs(a - b))) for a, b in pairs])
        edges = np.linspace(0.0, 0.58, 59)
        k = np.digitize(r, edges) - 1
        prof = np.array([out["rho"][k == i].mean() if np.any(k == i) else 0.0 for i in range(58)])
        i = int(np.argmax(prof))
        assert abs(0.5 * (edges[i] + edges[i + 1]) - sedov_radius(t)) < 2.0 * 1.2 / n_side + 0.01
    l1, l2 = np.array(l1), np.array(l2)
    print("Sedov t=0.1 L2 (rho, v_r, P) at 32^3, 64^3, 96^3:", l2.tolist(), " L1:", l1.tolist())
    for e in (l1, l2):
        assert np.all(e[1] < e[0]) and np.all(e[2] < e[1]), e
