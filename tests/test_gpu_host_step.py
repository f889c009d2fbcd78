"""sph_step_host (host buffers in and out, the copies inside the call) against sph_step on device
buffers: from the same converged state, the same steps must give the same bits in every field, with
pinned and with pageable host arrays, on one box and on a batch of boxes."""
import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig", "id")


def _converged(w, p, batch):
    from paper_2503_09713_gb300 import sph
    s = sph.DeviceState.from_numpy(w)
    solver = sph.Solver.batch(p, *batch) if batch else sph.Solver(p, w["n"])
    solver.converge(s)
    return solver, s


def _run(w, p, batch, pinned, steps=3):
    import torch
    from paper_2503_09713_gb300 import sph
    dev_solver, dev = _converged(w, p, batch)
    host_solver, src = _converged(w, p, batch)
    h = src.to_numpy()
    if pinned:   # page-locked copies of the host arrays
        for f in FIELDS:
            t = torch.empty(len(h[f]), dtype=torch.float64 if f != "id" else torch.int32, pin_memory=True)
            t.copy_(torch.from_numpy(h[f] if f != "id" else h[f].view(np.int32)))
            h[f] = t.numpy() if f != "id" else t.numpy().view(np.uint32)
    hst, arrs = sph.host_state({**h, "mass": w["mass"]})
    for _ in range(steps):
        a = dev_solver.step(dev)
        b = host_solver.step_host(hst)
        assert a == b
    out = dev.to_numpy()
    for f in FIELDS:
        assert np.array_equal(out[f], arrs[f]), f
    dev_solver.close()
    host_solver.close()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("precision", [0, 1])
def test_host_step_matches_device_step(precision, pinned):
    require_gpu()
    from paper_2503_09713_gb300 import sph, workloads
    w = workloads.lattice(16, sigma_v=0.05, seed=11)
    _run(w, sph.default_params(precision=precision), None, pinned)


def test_host_step_matches_device_step_on_a_batch():
    require_gpu()
    from paper_2503_09713_gb300 import replicas, sph, workloads
    boxes = workloads.ensemble(6, seed=5, n_min=512, n_max=4096)
    part = replicas.ensemble_shard(boxes, 1, 0)
    w = {**part["state"], "mass": 1.0}
    _run(w, sph.default_params(precision=1), (part["offsets"], part["mass"], part["gamma"]), True)
