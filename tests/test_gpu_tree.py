"""GPU tree build (App. B-C) against the oracle: bit-exact Morton codes, sort permutation, leaves,
Karras tables, tight boxes and h_max; the paper's worked examples through the GPU path."""
import numpy as np
import pytest

import oracle as O
from gpu_common import random_positions, require_gpu

pytestmark = pytest.mark.gpu


def _build(x, y, z, h, n_red, lo=(0, 0, 0), hi=(1, 1, 1), bits=21):
    require_gpu()
    from paper_2503_09713_gb300 import sph
    n = len(x)
    d = {"x": x, "y": y, "z": z, "h": h, "mass": 1.0 / n}
    s = sph.DeviceState.from_numpy(d)
    solver = sph.Solver(sph.default_params(reduction_level=n_red, box_lo=lo, box_hi=hi, morton_bits=bits), n)
    solver.build_tree(s)
    t = solver.export_tree()
    out = s.to_numpy()
    solver.close()
    return t, out


def expected_groups(leaf_first, tr, n):
    """Neighbour-search groups from the oracle's tree: the largest nodes holding at most 32
    particles, a leaf of more than 32 cut into runs of 32; returns the group starts and n."""
    L = len(leaf_first) - 1
    nin = L - 1

    def particles(t):
        if t < nin:
            e = int(tr.endrange[t])
            lo, hi = min(t, e), max(t, e)
        else:
            lo = hi = t - nin
        return int(leaf_first[lo]), int(leaf_first[hi + 1])

    starts, stack = [], [0]   # node 0: the root (internal, or the only leaf when L == 1)
    while stack:
        t = stack.pop()
        pf, pl = particles(t)
        if pl - pf <= 32:
            starts.append(pf)
        elif t >= nin:
            starts.extend(range(pf, pl, 32))
        else:
            stack.append(nin + int(tr.lchild[t]) if tr.lflag[t] else int(tr.lchild[t]))
            stack.append(nin + int(tr.rchild[t]) if tr.rflag[t] else int(tr.rchild[t]))
    return np.array(sorted(starts) + [n], dtype=np.int64)


def _check_against_oracle(x, y, z, h, n_red, lo=(0, 0, 0), hi=(1, 1, 1), bits=21):
    t, out = _build(x, y, z, h, n_red, lo, hi, bits)
    m = O.morton(x, y, z, lo, hi, bits=bits)
    mu, perm = O.sort_by_key(m)
    assert np.array_equal(t["mu"], mu)
    assert np.array_equal(t["perm"], perm)
    assert np.array_equal(out["id"], perm)
    xs, ys, zs, hs = x[perm], y[perm], z[perm], h[perm]
    assert np.array_equal(out["x"], xs) and np.array_equal(out["h"], hs)
    xi = O.keep_mask(mu, 3 * bits, n_red)
    idv, ml = O.compact(mu, xi)
    assert np.array_equal(t["leaf_first"], idv)
    assert np.array_equal(t["mu_leaf"], ml)
    tr = O.radix_tree(ml, 3 * bits)
    for k in ("lchild", "rchild", "lflag", "rflag", "endrange"):
        assert np.array_equal(t[k], getattr(tr, k)), k
    bmin, bmax, hmax = O.cell_boxes(idv, tr.endrange, xs, ys, zs, hs)
    assert np.array_equal(t["bmin"], bmin) and np.array_equal(t["bmax"], bmax) and np.array_equal(t["hmax"], hmax)
    assert np.array_equal(t["group_start"], expected_groups(idv, tr, len(x)))
    return len(ml)


@pytest.mark.parametrize("kind,n,n_red", [("uniform", 5000, 0), ("uniform", 5000, 3), ("cluster", 9001, 4),
                                          ("dups", 4099, 2), ("uniform", 70001, 3)])
def test_tree_bit_exact(kind, n, n_red):
    x, y, z = random_positions(n, 11 + n_red, kind)
    h = np.random.default_rng(5).uniform(0.01, 0.02, size=n)
    L = _check_against_oracle(x, y, z, h, n_red)
    assert 1 <= L <= n


@pytest.mark.parametrize("lo,hi", [((-0.6, -0.6, -0.6), (0.6, 0.6, 0.6)), ((-1.0, 0.0, 2.0), (1.0, 4.0, 2.5))])
def test_tree_other_boxes(lo, hi):
    """Boxes whose sides are not 1: span 1.2 (quotient path) and spans 2, 4, 0.5 (power-of-two path)."""
    x, y, z = random_positions(6000, 21, "uniform")
    lo, hi = np.array(lo), np.array(hi)
    x, y, z = [lo[k] + (hi[k] - lo[k]) * p for k, p in enumerate((x, y, z))]
    _check_against_oracle(x, y, z, np.full(6000, 0.05), 2, tuple(lo), tuple(hi))


@pytest.mark.parametrize("kind,n,n_red", [("uniform", 20000, 3), ("cluster", 9001, 2), ("dups", 4099, 1)])
def test_tree_u32_codes(kind, n, n_red):
    """The 30-bit codes of the u32 variant (10 bits per axis, App. B; 4 radix passes): codes,
    permutation, leaves, Karras tables, boxes and groups against the oracle at 10 bits."""
    x, y, z = random_positions(n, 31 + n_red, kind)
    h = np.random.default_rng(6).uniform(0.01, 0.02, size=n)
    _check_against_oracle(x, y, z, h, n_red, bits=10)


def test_tree_lattice_reduction_levels():
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(24, sigma_v=0.0, seed=99)
    counts = [_check_against_oracle(w["x"], w["y"], w["z"], w["h"], lv) for lv in range(0, 6)]
    assert counts[0] == 24 ** 3 and all(a > b for a, b in zip(counts, counts[1:]))


def test_tree_edge_sizes():
    for n in (1, 2, 3, 33):
        x, y, z = random_positions(n, n, "uniform")
        _check_against_oracle(x, y, z, np.full(n, 0.05), 3)
    # all particles on one point: a single leaf
    n = 100
    x = np.full(n, 0.3); y = np.full(n, 0.6); z = np.full(n, 0.9)
    t, _ = _build(x, y, z, np.full(n, 0.05), 2)
    assert list(t["leaf_first"]) == [0, n]
    assert list(t["group_start"]) == [0, 32, 64, 96, n]   # one leaf of 100 cut into runs of 32


def test_karras_table_through_gpu(golden):
    """Positions whose 63-bit codes start with the 6-bit codes of the Karras table example."""
    g = golden("karras_table.json")
    X, Y, Z = [], [], []
    for c in g["codes_6bit"]:
        v = int(c, 2)
        X.append(((v >> 5) & 1) * 2 + ((v >> 2) & 1))
        Y.append(((v >> 4) & 1) * 2 + ((v >> 1) & 1))
        Z.append(((v >> 3) & 1) * 2 + (v & 1))
    x = np.array(X) / 4 + 1 / 8
    y = np.array(Y) / 4 + 1 / 8
    z = np.array(Z) / 4 + 1 / 8
    t, _ = _build(x, y, z, np.full(12, 0.01), 0)
    assert [int(m >> np.uint64(57)) for m in t["mu_leaf"]] == [int(c, 2) for c in g["codes_6bit"]]
    assert list(t["lchild"]) == g["left_child_id"]
    assert list(t["rchild"]) == g["right_child_id"]
    assert list(t["lflag"]) == g["left_child_flag"]
    assert list(t["rflag"]) == g["right_child_flag"]
    assert list(t["endrange"]) == g["endrange"]


def test_mortonlistbuild_through_gpu(golden):
    g = golden("mortonlistbuild.json")
    codes = [int(c, 2) for c in g["m"]]
    x = np.array([(c >> 2) & 1 for c in codes]) * 0.5
    y = np.array([(c >> 1) & 1 for c in codes]) * 0.5
    z = np.array([c & 1 for c in codes]) * 0.5
    t, out = _build(x, y, z, np.full(7, 0.01), 0)
    assert [int(m >> np.uint64(60)) for m in t["mu"]] == [int(c, 2) for c in g["mu"]]
    assert list(t["leaf_first"]) == g["id"]
    assert [int(m >> np.uint64(60)) for m in t["mu_leaf"]] == [int(c, 2) for c in g["mu_leaf"]]
    m = np.array(codes)
    assert np.array_equal(m[t["perm"]], np.array([int(c, 2) for c in g["mu"]]))


@pytest.mark.parametrize("n_red", [5, 7])
def test_tree_reduction_across_tiles(n_red):
    """Many reduction passes over many 4096-code tiles of the one-launch reduction (each tile decides
    its codes from a halo of neighbouring codes): leaves bit-exact against the oracle."""
    x, y, z = random_positions(50000, 40 + n_red, "uniform")
    _check_against_oracle(x, y, z, np.full(50000, 0.01), n_red)


def test_tree_reduction_long_duplicate_runs():
    """Two runs of 2500 particles on one point each, inside a 30,000-particle set: the removed codes
    around them exceed any tile's halo, so those tiles take the pass-by-pass kernels; leaves stay
    bit-exact against the oracle."""
    x, y, z = random_positions(30000, 77, "uniform")
    x[:2500], y[:2500], z[:2500] = 0.31, 0.62, 0.93
    x[2500:5000], y[2500:5000], z[2500:5000] = 0.71, 0.22, 0.43
    _check_against_oracle(x, y, z, np.full(30000, 0.01), 4)
