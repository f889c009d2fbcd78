"""Parity at the sizes of the benchmark workloads, in the launch configuration bench.py times.

* uniform 32^3 (32,768 particles, FP64 and mixed): every particle against the oracle, for the
  converged initial state and for one full KDK step.
* Sedov 128^3 (2,097,152 particles, FP64, the benchmark workload): every particle against the
  oracle (uniform-grid candidates, OpenMP) for the tree, the converged state and one step;
  neighbour sets of sampled particles against brute force.
* uniform 256^3 (16,777,216 particles): mixed precision against FP64 for every particle
  (density <= 1e-5 relative, accelerations <= 1e-4 of max|a|), and 48 sampled particles of both
  runs against the oracle's definitions evaluated one by one (FP64 at the FP64 tolerances, mixed at
  the mixed ones).
* Sedov 512^3 (134,217,728 particles): the same checks on the converged state, and sampled
  particles after one FP64 step.

Tolerances as in test_gpu_physics (h: 1e-9 relative, from Newton's quadratic convergence after
|dh|/h <= 1e-6; accelerations on the same h: summation order only).
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import require_gpu, to_orig

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig")


def _orig(out):
    ids = out["id"].astype(np.int64)
    return {k: to_orig(out[k], ids) for k in FIELDS}


def _oracle_converged(w, P):
    h, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
    ax, ay, az, du, vs = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], h, om, w["mass"], P)
    st = {k: w[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    st.update(h=h, rho=rho, omega=om, ax=ax, ay=ay, az=az, du=du, vsig=vs)
    return st


def _compare_state(g, ref, precision, what):
    amax = np.max(np.abs(np.stack([ref["ax"], ref["ay"], ref["az"]])))
    if precision == 0:
        tol_h, tol_a, tol_rho = 1e-9, 1e-8 * amax, 3e-9
    else:
        tol_h, tol_a, tol_rho = 1e-5, 1e-4 * amax, 1e-5
    assert np.max(np.abs(g["h"] / ref["h"] - 1)) < tol_h, what + " h"
    assert np.max(np.abs(g["rho"] / ref["rho"] - 1)) < tol_rho, what + " rho"
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - ref[k])) < tol_a, what + " " + k
    dumax = np.max(np.abs(ref["du"]))
    assert np.max(np.abs(g["du"] - ref["du"])) < (1e-8 if precision == 0 else 1e-4) * dumax + 1e-300, what + " du"
    for k in ("x", "y", "z"):
        d = np.abs(g[k] - ref[k])
        assert np.max(np.minimum(d, 1.0 - d)) < 1e-13, what + " " + k


def _gpu_converged_and_step(w, ref0, precision, dt):
    from paper_2503_09713_gb300 import sph
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(sph.default_params(precision=precision), w["n"])
    solver.converge(s)
    g0 = _orig(s.to_numpy())
    # one step from the oracle's converged state, with the oracle's dt
    s1 = sph.DeviceState.from_numpy(dict(w, **{k: ref0[k] for k in ("h", "rho", "omega", "ax", "ay", "az", "du",
                                                                       "vsig")}))
    solver1 = sph.Solver(sph.default_params(precision=precision), w["n"])
    used, _ = solver1.step(s1, dt)
    g1 = _orig(s1.to_numpy())
    solver.close()
    solver1.close()
    return g0, g1


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform32_every_particle(precision):
    require_gpu()
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(32, sigma_v=0.01, seed=12345)
    P = O.Params()
    ref0 = _oracle_converged(w, P)
    dt = O.cfl(ref0["h"], ref0["vsig"], ref0["ax"], ref0["ay"], ref0["az"], P)
    ref1 = {k: v.copy() for k, v in ref0.items()}
    O.step(ref1, w["mass"], P, dt)
    g0, g1 = _gpu_converged_and_step(w, ref0, precision, dt)
    _compare_state(g0, ref0, precision, "converged")
    _compare_state(g1, ref1, precision, "after one step")


def test_sedov128_every_particle():
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.sedov(128, seed=12346)
    n = w["n"]
    P = O.Params()
    # tree at full size, bit-exact (default reduction level of the library)
    p = sph.default_params()
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(p, n)
    solver.build_tree(s)
    t = solver.export_tree()
    mu, perm = O.sort_by_key(O.morton(w["x"], w["y"], w["z"]))
    assert np.array_equal(t["mu"], mu) and np.array_equal(t["perm"], perm)
    xi = O.keep_mask(mu, 63, p.reduction_level)
    idv, ml = O.compact(mu, xi)
    assert np.array_equal(t["leaf_first"], idv)
    tr = O.radix_tree(ml, 63)
    for k in ("lchild", "rchild", "lflag", "rflag", "endrange"):
        assert np.array_equal(t[k], getattr(tr, k)), k
    bmin, bmax, hmax = O.cell_boxes(idv, tr.endrange, w["x"][perm], w["y"][perm], w["z"][perm], w["h"][perm])
    assert np.array_equal(t["bmin"], bmin) and np.array_equal(t["bmax"], bmax) and np.array_equal(t["hmax"], hmax)
    # neighbour sets of sampled particles (cache radius 2 chi max(h_a, h_b) at the initial h)
    solver.find_neighbours(s)
    off, ids = solver.export_neighbours(n)
    gid = s.to_numpy()["id"].astype(np.int64)
    rng = np.random.default_rng(3)
    rows = np.concatenate([rng.integers(0, n, 48), np.arange(16)])
    o_off, o_ids = O.subset_neighbours(w["x"], w["y"], w["z"], w["h"], 2.0 * 1.1, gid[rows])
    for k, a in enumerate(rows):
        assert np.array_equal(np.sort(gid[ids[off[a]:off[a + 1]]]), o_ids[o_off[k]:o_off[k + 1]])
    solver.close()
    # converged state and one step, every particle
    ref0 = _oracle_converged(w, P)
    dt = O.cfl(ref0["h"], ref0["vsig"], ref0["ax"], ref0["ay"], ref0["az"], P)
    ref1 = {k: v.copy() for k, v in ref0.items()}
    O.step(ref1, w["mass"], P, dt)
    g0, g1 = _gpu_converged_and_step(w, ref0, 0, dt)
    _compare_state(g0, ref0, 0, "converged")
    _compare_state(g1, ref1, 0, "after one step")


def test_uniform256_mixed_against_fp64_and_sampled_oracle():
    torch = require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(256, sigma_v=0.1, seed=12347)
    n = w["n"]
    out = {}
    for precision in (0, 1):
        s = sph.DeviceState.from_numpy(w)
        solver = sph.Solver(sph.default_params(precision=precision), n)
        solver.converge(s)
        out[precision] = _orig(s.to_numpy())
        solver.close()
        del s
        torch.cuda.empty_cache()
    g64, g32 = out[0], out[1]
    assert np.max(np.abs(g32["rho"] / g64["rho"] - 1)) < 1e-5
    amax = np.max(np.abs(np.stack([g64["ax"], g64["ay"], g64["az"]])))
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g32[k] - g64[k])) < 1e-4 * amax
    # sampled particles of both runs against the definitions, evaluated one by one on the
    # neighbourhood of the samples (exact: see _local): FP64 at the FP64 tolerances, mixed at the
    # mixed ones (density 1e-5 relative, accelerations 1e-4 of max|a|)
    rng = np.random.default_rng(9)
    idx = rng.choice(n, 48, replace=False)
    h_hi = 2.0 * w["dx"]   # h is ~1.2 dx; a root above this bound raises in the oracle
    cells = _CellIndex(w, 4.2 * h_hi)
    rs = []
    for a in idx:
        sub, j = cells.local(a)
        rs.append(O.subset_forces(*[sub[k] for k in ("x", "y", "z", "vx", "vy", "vz", "u")], w["mass"],
                                  O.Params(), [j], h_hi))
    r = {k: np.array([x[k][0] for x in rs]) for k in rs[0]}
    assert np.max(np.abs(g64["h"][idx] / r["h"] - 1)) < 1e-9
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g64[k][idx] - r[k])) < 1e-8 * amax
    rho_o = w["mass"] * (1.2 / r["h"]) ** 3
    assert np.max(np.abs(g32["rho"][idx] / rho_o - 1)) < 1e-5
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g32[k][idx] - r[k])) < 1e-4 * amax


def _fetch(s, fields):
    """Selected fields of a device state, in the original particle order (host copies)."""
    ids = s.t["id"].cpu().numpy().view(np.uint32).astype(np.int64)
    return {f: to_orig(s.t[f].cpu().numpy(), ids) for f in fields}


class _CellIndex:
    """Particles of a periodic unit box binned into cells of side >= radius: the particles within
    `radius` of one particle, as sub-arrays, from its 27 surrounding cells (see _local for why such
    a neighbourhood gives the oracle's exact answer when radius is above 4 h_hi)."""

    def __init__(self, st, radius):
        self.st, self.r = st, radius
        self.G = G = max(3, int(1.0 / radius))
        self.c = [np.minimum((st[k] * G).astype(np.int64), G - 1) for k in ("x", "y", "z")]
        key = (self.c[0] * G + self.c[1]) * G + self.c[2]
        self.order = np.argsort(key, kind="stable")
        self.skey = key[self.order]

    def local(self, a):
        G, st = self.G, self.st
        ca = [int(c[a]) for c in self.c]
        parts = []
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for oz in (-1, 0, 1):
                    key = (((ca[0] + ox) % G) * G + (ca[1] + oy) % G) * G + (ca[2] + oz) % G
                    lo, hi = np.searchsorted(self.skey, [key, key + 1])
                    parts.append(self.order[lo:hi])
        sel = np.unique(np.concatenate(parts))
        d2 = np.zeros(len(sel))
        for k in ("x", "y", "z"):
            d = np.abs(st[k][sel] - st[k][a])
            d = np.minimum(d, 1.0 - d)
            d2 += d * d
        sel = sel[d2 < self.r * self.r]
        sub = {k: np.ascontiguousarray(st[k][sel]) for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
        return sub, int(np.searchsorted(sel, a))


def _local(st, idx, radius):
    """The particles within `radius` (periodic unit box) of any particle in idx, as sub-arrays, and
    the positions of idx in them.  The oracle's answer for a particle depends only on particles
    within 2 * (2 h_hi) of it, so evaluating it on this neighbourhood (radius above 4 h_hi) is
    exact and avoids its O(n) candidate scans over 134 M particles."""
    keep = np.zeros(len(st["x"]), dtype=bool)
    for a in idx:
        d2 = np.zeros(len(st["x"]))
        for k in ("x", "y", "z"):
            d = np.abs(st[k] - st[k][a])
            d = np.minimum(d, 1.0 - d)
            d2 += d * d
        keep |= d2 < radius * radius
    sel = np.flatnonzero(keep)
    sub = {k: np.ascontiguousarray(st[k][sel]) for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    return sub, np.searchsorted(sel, idx)


def test_sedov512_sampled_and_mixed_against_fp64():
    """Sedov 512^3 (134,217,728 particles), the largest configuration, in the launch configuration
    bench.py uses: FP64 converged state and the state after one CFL step on sampled particles
    (blast and background) against the oracle's definitions evaluated one by one; the mixed
    path against FP64 for every particle."""
    torch = require_gpu()
    if torch.cuda.mem_get_info()[1] < 200e9:
        pytest.skip("needs a GPU with more than 200 GB")
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.sedov(512, seed=12346)
    n = w["n"]
    P = O.Params()
    h_hi = 1.5 * w["dx"]   # the density stays within a few per cent of the lattice's in one step
    rng = np.random.default_rng(11)
    idx = np.concatenate([rng.choice(np.flatnonzero(w["u"] > 1e-6), 3, replace=False), rng.integers(0, n, 3)])
    state_fields = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du")
    got = {}
    for precision in (0, 1):
        s = sph.DeviceState.from_numpy(w)
        solver = sph.Solver(sph.default_params(precision=precision), n)
        solver.converge(s)
        got[precision] = _fetch(s, ("h", "rho", "ax", "ay", "az", "du"))
        if precision == 0:
            used, _ = solver.step(s, 0.0)
            assert used > 0
            after = _fetch(s, state_fields)
        solver.close()
        del s, solver
        torch.cuda.empty_cache()
    g64, g32 = got[0], got[1]
    amax = np.max(np.abs(np.stack([g64["ax"], g64["ay"], g64["az"]])))
    sub, j = _local(w, idx, 4.5 * h_hi)
    r = O.subset_forces(*[sub[k] for k in ("x", "y", "z", "vx", "vy", "vz", "u")], w["mass"], P, j, h_hi)
    assert np.max(np.abs(g64["h"][idx] / r["h"] - 1)) < 1e-9
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g64[k][idx] - r[k])) < 1e-8 * amax, k
    assert np.max(np.abs(g32["rho"] / g64["rho"] - 1)) < 1e-5
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g32[k] - g64[k])) < 1e-4 * amax, k
    # after the step the state holds v^{n+1}, u^{n+1}; its accelerations were evaluated at the
    # predicted v* = v^{n+1} - dt/2 (a^{n+1} - a^n) and u* likewise (App. G), so the oracle gets those
    hdt = 0.5 * used
    mid = dict(after)
    for v, a in (("vx", "ax"), ("vy", "ay"), ("vz", "az"), ("u", "du")):
        mid[v] = after[v] - hdt * (after[a] - g64[a])
    sub1, j1 = _local(mid, idx, 4.5 * h_hi)
    r1 = O.subset_forces(*[sub1[k] for k in ("x", "y", "z", "vx", "vy", "vz", "u")], w["mass"], P, j1, h_hi)
    amax1 = np.max(np.abs(np.stack([after["ax"], after["ay"], after["az"]])))
    assert np.max(np.abs(after["h"][idx] / r1["h"] - 1)) < 1e-9
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(after[k][idx] - r1[k])) < 1e-8 * amax1, k
