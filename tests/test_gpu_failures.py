"""Failure detection on the device, in forms that fault or hang nothing.

* A bounded device-side wait that runs out (a look-back word that nothing publishes) returns
  SPH_ERR_TIMEOUT and leaves the context usable: the radix-sort look-back and the stage-2 look-back,
  each made to run out by the library's probe (sph_debug_wait_timeout) after a few thousand rounds.
* A NaN or infinite position, or a smoothing length <= 0, gives SPH_ERR_NONFINITE from the tree build.
* The Newton iteration of App. F capped at one iteration, from h 5% above the root, gives
  SPH_ERR_H_NOT_CONVERGED (the iteration cap of the paper's inner loop).
Every check ends with a normal call on the same context that must succeed and match a fresh one.
"""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _solver(w, **kw):
    from paper_2503_09713_gb300 import sph
    s = sph.DeviceState.from_numpy(w)
    return sph, s, sph.Solver(sph.default_params(**kw), w["n"])


def test_sort_lookback_timeout_is_reported():
    require_gpu()
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(16, seed=3)
    sph, s, solver = _solver(w)
    for spins in (1, 4096):
        code = sph.sph_debug_wait_timeout(solver.ctx, s.c(), 0, spins)
        assert code == sph.SPH_ERR_TIMEOUT, code
    solver.build_tree(s)                         # the context still works
    t = solver.export_tree()
    assert np.all(np.diff(t["mu"].astype(np.float64)) >= 0)
    solver.close()


def test_stage2_lookback_timeout_is_reported_and_cache_rebuilds():
    require_gpu()
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(16, seed=4)
    sph, s, solver = _solver(w)
    solver.build_tree(s)
    solver.find_neighbours(s)
    off0, ids0 = solver.export_neighbours(w["n"])
    code = sph.sph_debug_wait_timeout(solver.ctx, s.c(), 1, 4096)
    assert code == sph.SPH_ERR_TIMEOUT, code
    with pytest.raises(sph.SPHError) as e:       # the probe invalidated the cache
        solver.compute_density_h(s)
    assert e.value.code == sph.SPH_ERR_ORDER
    solver.find_neighbours(s)
    off1, ids1 = solver.export_neighbours(w["n"])
    assert np.array_equal(off0, off1) and np.array_equal(ids0, ids1)
    solver.compute_density_h(s)
    solver.close()


@pytest.mark.parametrize("field,value", [("x", np.nan), ("z", np.inf), ("h", 0.0), ("h", np.nan)])
def test_nonfinite_input_is_reported(field, value):
    require_gpu()
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(12, seed=5)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in w.items()}
    bad[field][37] = value
    sph, s, solver = _solver(bad)
    with pytest.raises(sph.SPHError) as e:
        solver.build_tree(s)
    assert e.value.code == sph.SPH_ERR_NONFINITE
    solver.close()
    # a good state on a new context afterwards
    sph, s2, solver2 = _solver(w)
    solver2.converge(s2)
    solver2.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_iteration_cap_is_reported(precision):
    require_gpu()
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(12, seed=6)
    sph, s, solver = _solver(w, precision=precision)
    solver.converge(s)
    conv = s.to_numpy()
    solver.close()
    start = dict(w)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "id"):
        start[k] = conv[k]
    start["h"] = 1.05 * conv["h"]               # Newton moves h down by ~5%: inside the cache tolerance
    sph, s1, capped = _solver(start, precision=precision, h_max_iter=1)
    capped.build_tree(s1)
    capped.find_neighbours(s1)
    with pytest.raises(sph.SPHError) as e:
        capped.compute_density_h(s1)
    assert e.value.code == sph.SPH_ERR_H_NOT_CONVERGED
    capped.close()
    sph, s2, free = _solver(start, precision=precision)
    free.build_tree(s2)
    free.find_neighbours(s2)
    assert free.compute_density_h(s2) > 1       # more than one iteration was needed
    free.close()
