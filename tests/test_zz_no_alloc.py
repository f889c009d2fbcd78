"""The allocation-free Morton sort (sph_sort_morton_noalloc) against the oracle.

Some callers cannot allocate device memory (their memory belongs to another allocator, or they
cannot take the synchronisation of cudaFree), so this entry point keeps its scratch in a fixed
device array inside the library.  This file is collected last on purpose.  The check: two calls in
a row on each input, each compared bit for bit with the oracle's Morton codes (App. B) and stable
sort (App. C), at the size limit (n = 262144, 64 sort tiles), on a box that is not the unit box, and
with duplicate codes; the regular tree build's export must agree as well."""
import numpy as np
import pytest

import oracle as O
from gpu_common import random_positions, require_gpu

pytestmark = pytest.mark.gpu


def _tree_export(x, y, z, lo, hi):
    from paper_2503_09713_gb300 import sph
    n = len(x)
    p = sph.default_params(box_lo=lo, box_hi=hi)
    s = sph.DeviceState.from_numpy({"x": x, "y": y, "z": z, "h": np.full(n, 1e-3 * (hi[0] - lo[0])),
                                    "mass": 1.0 / n})
    solver = sph.Solver(p, n)
    solver.build_tree(s)
    t = solver.export_tree()
    solver.close()
    return t["mu"], t["perm"]


def _noalloc(torch, x, y, z, lo, hi):
    from paper_2503_09713_gb300 import sph
    n = len(x)
    dev = [torch.from_numpy(a).cuda() for a in (x, y, z)]
    codes = torch.zeros(n, dtype=torch.int64, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    sph.sph_sort_morton_noalloc(n, dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr(), lo, hi,
                                codes.data_ptr(), perm.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return codes.cpu().numpy().view(np.uint64), perm.cpu().numpy().view(np.uint32)


CASES = [
    (262144, 1, "uniform", (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)),       # the limit: 64 full tiles
    (70001, 2, "dups", (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)),            # equal codes: stability
    (100003, 3, "cluster", (-0.5, 0.25, 2.0), (1.5, 1.0, 5.0)),      # non-unit box, ragged tail
]


def test_noalloc_sort_matches_oracle_twice():
    torch = require_gpu()
    for n, seed, kind, lo, hi in CASES:
        x, y, z = random_positions(n, seed, kind)
        lo_a, hi_a = np.array(lo), np.array(hi)
        x, y, z = (lo_a[k] + (hi_a[k] - lo_a[k]) * c for k, c in enumerate((x, y, z)))
        mu_ref, perm_ref = O.sort_by_key(O.morton(x, y, z, lo=lo, hi=hi, bits=21))
        for _ in range(2):
            mu, perm = _noalloc(torch, x, y, z, lo, hi)
            assert np.array_equal(mu, mu_ref), (n, kind)
            assert np.array_equal(perm, perm_ref), (n, kind)
        mu_t, perm_t = _tree_export(x, y, z, lo, hi)
        assert np.array_equal(mu_t, mu_ref) and np.array_equal(perm_t, perm_ref)


def test_noalloc_sort_sizes():
    torch = require_gpu()
    from paper_2503_09713_gb300 import sph
    with pytest.raises(sph.SPHError) as e:
        sph.sph_sort_morton_noalloc(262145, 1, 1, 1, (0, 0, 0), (1, 1, 1), 1, 1)
    assert e.value.code == sph.SPH_ERR_CAPACITY
    with pytest.raises(sph.SPHError) as e:
        sph.sph_sort_morton_noalloc(-1, 1, 1, 1, (0, 0, 0), (1, 1, 1), 1, 1)
    assert e.value.code == sph.SPH_ERR_INVALID_ARG
    # n = 0 succeeds and writes nothing
    codes = torch.full((4,), 7, dtype=torch.int64, device="cuda")
    sph.sph_sort_morton_noalloc(0, 1, 1, 1, (0, 0, 0), (1, 1, 1), codes.data_ptr(), 1,
                                torch.cuda.current_stream().cuda_stream)
    assert codes.cpu().tolist() == [7, 7, 7, 7]
