"""Launch shapes (sph_set_launch) and the autotuner (sph_autotune): results do not depend on the
shapes, and the tuned context still matches the oracle."""
import numpy as np
import pytest

import oracle as O
from gpu_common import require_gpu, to_orig

pytestmark = pytest.mark.gpu

OUT = ("h", "rho", "omega", "ax", "ay", "az", "du", "vsig")


def _orig(s):
    d = s.to_numpy()
    ids = d["id"].astype(np.int64)
    return {k: to_orig(d[k], ids) for k in OUT}


@pytest.mark.parametrize("precision", [0, 1])
def test_results_independent_of_launch_shapes(precision):
    """Same input state, different block sizes / stage-2 warps / reduction levels: identical
    neighbour sets and bit-identical h, rho, Omega, a, du, v_sig."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.sedov(20, seed=31)
    ref = None
    for shape in (dict(density_block=128, forces_block=128, walk_block=128, stage2_warps=4, reduction_level=3),
                  dict(density_block=64, forces_block=256, walk_block=64, stage2_warps=1, reduction_level=1),
                  dict(density_block=256, forces_block=64, walk_block=256, stage2_warps=8, reduction_level=5)):
        s = sph.DeviceState.from_numpy(w)
        solver = sph.Solver(sph.default_params(precision=precision), w["n"])
        solver.set_launch(**shape)
        assert solver.launch() == shape
        solver.converge(s)
        out = _orig(s)
        solver.close()
        if ref is None:
            ref = out
        else:
            for k in OUT:
                assert np.array_equal(out[k], ref[k]), (shape, k)


def test_set_launch_rejects_bad_shapes():
    require_gpu()
    from paper_2503_09713_gb300 import sph
    solver = sph.Solver(sph.default_params(), 1000)
    for bad in (dict(density_block=96), dict(forces_block=512), dict(stage2_warps=0), dict(stage2_warps=9),
                dict(reduction_level=-1)):
        with pytest.raises(sph.SPHError):
            solver.set_launch(**bad)
    solver.close()


def test_autotune_then_oracle():
    """The autotuner returns a valid shape, leaves a converged state (h moved by less than h_tol h)
    and the context keeps matching the oracle for a KDK step."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(24, sigma_v=0.1, jitter=0.1, seed=41)
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver(sph.default_params(), w["n"])
    solver.converge(s)
    before = _orig(s)
    best, ms = solver.autotune(s)
    assert ms > 0 and best == solver.launch()
    assert best["density_block"] in (64, 128, 256) and 1 <= best["stage2_warps"] <= 8
    assert 1 <= best["reduction_level"] <= 7
    after = _orig(s)
    assert np.max(np.abs(after["h"] / before["h"] - 1)) < 1e-6
    P = O.Params()
    amax = np.max(np.abs(np.stack([before["ax"], before["ay"], before["az"]])))
    d = s.to_numpy()
    ids = d["id"].astype(np.int64)
    st = {k: to_orig(d[k], ids) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho",
                                           "omega", "vsig")}
    dt = O.cfl(st["h"], st["vsig"], st["ax"], st["ay"], st["az"], P)
    ref = {k: v.copy() for k, v in st.items()}
    O.step(ref, w["mass"], P, dt)
    used, _ = solver.step(s, dt)
    assert used == dt
    g = _orig(s)
    assert np.max(np.abs(g["h"] / ref["h"] - 1)) < 1e-9
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - ref[k])) < 1e-8 * amax, k
    solver.close()
