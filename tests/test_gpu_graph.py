"""Graph replay of sph_step (sph_set_graph): a step recorded once into a CUDA graph and replayed must
give the same bits as the stage-by-stage step, on one box and on a batch, and must finish on the host
path when a count outgrows its arrays or h leaves the cache tolerance."""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig", "id")


def _pair(w, p, batch=None):
    """Two solvers on copies of the same state: graph replay on, and off."""
    from paper_2503_09713_gb300 import sph
    out = []
    for graph in (True, False):
        s = sph.DeviceState.from_numpy(w)
        solver = sph.Solver.batch(p, *batch) if batch else sph.Solver(p, w["n"])
        solver.set_graph(graph)
        solver.converge(s)
        out.append((solver, s))
    return out


def _same(a, b, what):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), (what, k)
    if "alpha" in a:
        assert np.array_equal(a["alpha"], b["alpha"]), (what, "alpha")


def _steps(pair, n, dt=0.0):
    dts = []
    for solver, s in pair:
        d = []
        for _ in range(n):
            used, nxt = solver.step(s, dt)
            d.append((used, nxt))
        dts.append(d)
    assert dts[0] == dts[1]


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_step_is_bit_identical(precision):
    """Jittered 20^3 lattice, 6 CFL steps: every field, the particle order and the time steps agree
    bit for bit; the first step runs stage by stage, the second captures, the rest replay."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(20, sigma_v=0.1, jitter=0.1, seed=31)
    pair = _pair(w, sph.default_params(precision=precision))
    _steps(pair, 6)
    _same(pair[0][1].to_numpy(), pair[1][1].to_numpy(), "lattice")
    st = pair[0][0].stats()
    assert st["graph_captures"] == 1 and st["graph_replays"] == 5 and st["graph_fallbacks"] == 0, st
    assert pair[1][0].stats()["graph_replays"] == 0
    for k in ("n_leaves", "n_groups", "n_pairs", "cache_slots", "cand_chunks", "density_iters_max",
              "density_pair_evals", "force_pairs", "dt_next"):
        assert st[k] == pair[1][0].stats()[k], k


def test_graph_step_with_switch_and_corrector_reruns():
    """Sedov blast with the shock switch, per-particle alpha and the corrector check (re-runs after the
    replayed first pass): bit-identical to the stage-by-stage steps."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.sedov(16, seed=5, hfact=1.2)
    w["alpha"] = np.full(w["n"], 1.0)
    p = sph.default_params(av_switch=1, eps_v=1e-3, max_corr=3)
    pair = _pair(w, p)
    _steps(pair, 5)
    _same(pair[0][1].to_numpy(), pair[1][1].to_numpy(), "sedov")
    a, b = pair[0][0].stats(), pair[1][0].stats()
    assert a["graph_replays"] >= 3 and a["cfl_multiplier"] == b["cfl_multiplier"], (a, b)


def test_graph_batch_is_bit_identical():
    """Ensemble of 12 boxes of uneven sizes, mixed precision, per-box CFL steps."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    boxes = workloads.ensemble(12, seed=9, n_min=512, n_max=6000)
    off = np.concatenate([[0], np.cumsum([b["n"] for b in boxes])]).astype(np.int64)
    cat = {k: np.concatenate([b[k] for b in boxes]) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h")}
    cat["mass"] = 1.0
    cat["n"] = int(off[-1])
    pair = _pair(cat, sph.default_params(precision=sph.SPH_MIXED),
                 (off, np.array([b["mass"] for b in boxes]), np.array([b["gamma"] for b in boxes])))
    _steps(pair, 5)
    _same(pair[0][1].to_numpy(), pair[1][1].to_numpy(), "ensemble")
    assert np.array_equal(pair[0][0].batch_dt(), pair[1][0].batch_dt())
    assert pair[0][0].stats()["graph_replays"] == 4


def test_graph_falls_back_when_the_cache_outgrows_its_arrays():
    """After three replays every h is doubled in place (eight times the neighbours inside the cache
    radius): the replay finds the candidate lists and the cache too small, the host finishes that
    step stage by stage with grown arrays (the h iteration brings h back down), the next step
    captures again, and every result still equals the stage-by-stage run given the same change."""
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(16, sigma_v=0.05, jitter=0.1, seed=44)
    pair = _pair(w, sph.default_params())
    _steps(pair, 4, dt=2e-4)
    for solver, s in pair:
        s.t["h"].mul_(2.0)
    _steps(pair, 3, dt=2e-4)
    _same(pair[0][1].to_numpy(), pair[1][1].to_numpy(), "h doubled")
    st = pair[0][0].stats()
    assert st["graph_fallbacks"] >= 1 and st["graph_captures"] >= 2, st
