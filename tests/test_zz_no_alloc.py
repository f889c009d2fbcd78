"""The allocation-free Morton sort (sph_sort_morton_noalloc) against the regular tree build.

Some callers cannot allocate device memory (their memory belongs to another allocator, or they
cannot take the synchronisation of cudaFree), so this entry point keeps its scratch in a fixed
device array inside the library.  This file is collected last on purpose.  The check: two calls in
a row, each compared with the codes and permutation that sph_build_tree exports for the same
positions (integers: bit-exact)."""
import numpy as np
import pytest

from gpu_common import random_positions, require_gpu

pytestmark = pytest.mark.gpu


def _reference(x, y, z):
    from paper_2503_09713_gb300 import sph
    n = len(x)
    s = sph.DeviceState.from_numpy({"x": x, "y": y, "z": z, "h": np.full(n, 0.01), "mass": 1.0 / n})
    solver = sph.Solver(sph.default_params(), n)
    solver.build_tree(s)
    t = solver.export_tree()
    solver.close()
    return t["mu"], t["perm"]


def _noalloc(torch, x, y, z):
    from paper_2503_09713_gb300 import sph
    n = len(x)
    dev = [torch.from_numpy(a).cuda() for a in (x, y, z)]
    codes = torch.zeros(n, dtype=torch.int64, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    sph.sph_sort_morton_noalloc(n, dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr(), (0, 0, 0), (1, 1, 1),
                                codes.data_ptr(), perm.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return codes.cpu().numpy().view(np.uint64), perm.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_tree_build_twice():
    torch = require_gpu()
    for n, seed, kind in ((200000, 1, "uniform"), (70001, 2, "dups")):
        x, y, z = random_positions(n, seed, kind)
        mu_ref, perm_ref = _reference(x, y, z)
        mu, perm = _noalloc(torch, x, y, z)
        assert np.array_equal(mu, mu_ref)
        assert np.array_equal(perm, perm_ref)


def test_noalloc_sort_rejects_oversize():
    require_gpu()
    from paper_2503_09713_gb300 import sph
    with pytest.raises(sph.SPHError) as e:
        sph.sph_sort_morton_noalloc(262145, 1, 1, 1, (0, 0, 0), (1, 1, 1), 1, 1)
    assert e.value.code == sph.SPH_ERR_CAPACITY
