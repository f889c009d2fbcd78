"""GPU neighbour cache (App. C two-stage cache, App. D criteria) against the definition: for every
particle the set {b != a : r_ab^2 < (2 chi max(h_a, h_b))^2} (nearest periodic image), bit-exact."""
import numpy as np
import pytest

import oracle as O
from gpu_common import random_positions, require_gpu, to_orig

pytestmark = pytest.mark.gpu


def _gpu_sets(d, params):
    require_gpu()
    from paper_2503_09713_gb300 import sph
    s = sph.DeviceState.from_numpy(d)
    solver = sph.Solver(params, len(d["x"]))
    solver.build_tree(s)
    npairs = solver.find_neighbours(s)
    off, ids = solver.export_neighbours(len(d["x"]))
    out = s.to_numpy()
    solver.close()
    return out["id"].astype(np.int64), off, ids, npairs


def _compare(d, n_red=3, chi=1.1, periodic=1):
    from paper_2503_09713_gb300 import sph
    p = sph.default_params(reduction_level=n_red, cache_tol=chi, periodic=periodic)
    gid, off, ids, npairs = _gpu_sets(d, p)
    o_off, o_ids = O.neighbours(d["x"], d["y"], d["z"], d["h"], 2.0 * chi, periodic=periodic, method=0)
    n = len(d["x"])
    assert npairs == len(o_ids) == off[-1]
    for a in range(n):
        ga = gid[a]
        got = np.sort(gid[ids[off[a]:off[a + 1]]])
        exp = o_ids[o_off[ga]:o_off[ga + 1]]
        assert np.array_equal(got, exp), f"particle {ga}"


@pytest.mark.parametrize("kind,n", [("uniform", 3001), ("cluster", 4000), ("dups", 2049)])
def test_sets_equal_definition(kind, n):
    x, y, z = random_positions(n, 3, kind)
    rng = np.random.default_rng(4)
    h = rng.uniform(0.02, 0.045, size=n) if kind != "cluster" else rng.uniform(0.01, 0.06, size=n)
    _compare({"x": x, "y": y, "z": z, "h": h, "mass": 1.0 / n})


@pytest.mark.parametrize("n_red", [0, 1, 5])
def test_sets_lattice_reduction_levels(n_red):
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(14, sigma_v=0.0, jitter=0.2, seed=2)
    _compare(w, n_red=n_red)


def test_sets_open_box_and_sedov_like_h():
    from paper_2503_09713_gb300 import workloads
    w = workloads.sedov(14)
    r = np.sqrt((w["x"] - 0.5) ** 2 + (w["y"] - 0.5) ** 2 + (w["z"] - 0.5) ** 2)
    w["h"] = w["h"] * (1.0 + 2.0 * np.exp(-(r / 0.15) ** 2))     # large h in the centre, as after the blast
    _compare(w)
    _compare(w, periodic=0)


def test_exact_band_on_lattice():
    """Perfect lattice: many pairs sit exactly at lattice distances; the FP64 decision must hold for
    neighbours placed exactly on the radius (2 chi h = sqrt(5) dx here)."""
    from paper_2503_09713_gb300 import workloads
    w = workloads.perfect_lattice(16)
    w["h"][:] = np.sqrt(5.0) * w["dx"] / 2.2
    _compare(w)
