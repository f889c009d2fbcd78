"""Pins of the oracle's tree functions (App. B-C) against the paper's worked examples and invariants."""
import numpy as np
import pytest

import oracle as O


def b2i(s):
    return int(s, 2)


def test_prefix_worked_example(golden):
    """Eqs. delta_ab / hat / ex and the mask/prefix example of App. B."""
    g = golden("morton_prefix.json")
    m1, m2, nb = b2i(g["m1"]), b2i(g["m2"]), g["nbits"]
    assert m1 ^ m2 == b2i(g["xor"])
    d = O.delta(m1, m2, nb)
    assert d == g["delta"]
    mask = (((1 << nb) - 1) << (nb - d)) & ((1 << nb) - 1)
    assert mask == b2i(g["mask"])
    assert (m2 & mask) == b2i(g["prefix"])


def test_morton_round_trip_exhaustive():
    """Interleaving is a bijection on a 3-bit-per-axis grid, x most significant."""
    seen = set()
    for X in range(8):
        for Y in range(8):
            for Z in range(8):
                m = O.interleave(X, Y, Z, 3)
                assert O.deinterleave(m, 3) == (X, Y, Z)
                seen.add(m)
    assert seen == set(range(512))
    # x is the most significant bit of each triplet
    assert O.interleave(1, 0, 0, 1) == 0b100
    assert O.interleave(0, 1, 0, 1) == 0b010
    assert O.interleave(0, 0, 1, 1) == 0b001


def test_morton_octant_and_quantise():
    """The first triplet of a code is the octant (App. B: X0 = 1 iff X in the upper half)."""
    rng = np.random.default_rng(1)
    p = rng.uniform(0, 1, size=(500, 3))
    m = O.morton(p[:, 0], p[:, 1], p[:, 2], bits=21)
    top = (m >> np.uint64(60)).astype(np.int64)
    expect = (p[:, 0] >= 0.5) * 4 + (p[:, 1] >= 0.5) * 2 + (p[:, 2] >= 0.5) * 1
    assert np.array_equal(top, expect)
    assert O.quantise(1.0, 0.0, 1.0, 21) == (1 << 21) - 1      # upper face joins the last cell
    assert O.quantise(-1e-300, 0.0, 1.0, 21) == 0
    assert O.quantise(0.5, 0.0, 1.0, 21) == 1 << 20


def test_sort_stable():
    keys = np.array([5, 3, 5, 1, 3, 3], np.uint64)
    s, perm = O.sort_by_key(keys)
    assert list(s) == [1, 3, 3, 3, 5, 5]
    assert list(perm) == [3, 1, 4, 5, 0, 2]


def test_mortonlistbuild_figure(golden):
    """Fig. mortonlistbuild: sort, duplicate mask, compaction, leaf codes."""
    g = golden("mortonlistbuild.json")
    m = np.array([b2i(c) for c in g["m"]], np.uint64)
    mu, perm = O.sort_by_key(m)
    assert [int(v) for v in mu] == [b2i(c) for c in g["mu"]]
    assert np.array_equal(m[perm], mu)
    xi = O.keep_mask(mu, g["nbits"], 0)
    assert list(xi) == g["xi"]
    idv, ml = O.compact(mu, xi)
    assert list(idv) == g["id"]
    assert [int(v) for v in ml] == [b2i(c) for c in g["mu_leaf"]]


def test_karras_table(golden):
    """Table arrays_fig_karras, reproduced by the oracle's top-down definition of the tree."""
    g = golden("karras_table.json")
    codes = np.array([b2i(c) for c in g["codes_6bit"]], np.uint64)
    t = O.radix_tree(codes, g["nbits"])
    assert list(t.lchild) == g["left_child_id"]
    assert list(t.rchild) == g["right_child_id"]
    assert list(t.lflag) == g["left_child_flag"]
    assert list(t.rflag) == g["right_child_flag"]
    assert list(t.endrange) == g["endrange"]


def _tree_invariants(codes, nbits, t):
    """Structural invariants of a binary radix tree over L sorted distinct codes."""
    L = len(codes)
    n_in = L - 1
    parent_count = np.zeros(2 * L - 1, np.int64)
    for i in range(n_in):
        for cid, fl in ((t.lchild[i], t.lflag[i]), (t.rchild[i], t.rflag[i])):
            node = cid + n_in if fl else cid
            parent_count[node] += 1
        lo, hi = min(i, t.endrange[i]), max(i, t.endrange[i])
        d_node = O.delta(int(codes[lo]), int(codes[hi]), nbits)
        # every code inside the range shares the node prefix; the neighbours outside do not extend it
        for k in range(lo, hi + 1):
            assert O.delta(int(codes[lo]), int(codes[k]), nbits) >= d_node
        if lo > 0:
            assert O.delta(int(codes[lo - 1]), int(codes[lo]), nbits) < d_node
        if hi < L - 1:
            assert O.delta(int(codes[hi]), int(codes[hi + 1]), nbits) < d_node
    assert parent_count[0] == 0                       # root
    assert np.all(parent_count[1:] == 1)               # every other node has one parent


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_radix_tree_random_invariants(seed):
    rng = np.random.default_rng(seed)
    codes = np.unique(rng.integers(0, 1 << 20, size=300, dtype=np.uint64))
    t = O.radix_tree(codes, 20)
    _tree_invariants(codes, 20, t)


def _delta_rule_pass(codes, nbits):
    """One reduction pass stated through prefix lengths of neighbouring kept codes (the comparison
    form of App. C's listing, written here independently of the oracle, which works on the radix
    tree): code j is dropped when delta(j-1, j) exceeds both delta(j-2, j-1) and delta(j, j+1), a
    neighbour missing at either end counting as -1.  Returns the kept flags."""
    L = len(codes)
    c = [int(v) for v in codes]

    def d(i, j):
        if i < 0 or j >= L:
            return -1
        return nbits - (c[i] ^ c[j]).bit_length()

    return [not (j >= 1 and d(j - 1, j) > d(j - 2, j - 1) and d(j - 1, j) > d(j, j + 1)) for j in range(L)]


@pytest.mark.parametrize("seed", [3, 4])
def test_reduction_matches_prefix_comparison_rule(seed):
    """App. C 'Reduction': the oracle removes the second leaf of every leaf-leaf sibling pair of the
    radix tree; the same passes stated as comparisons of neighbouring prefix lengths must agree,
    level by level, on random codes with duplicates."""
    rng = np.random.default_rng(seed)
    nbits = 30
    raw = np.sort(rng.integers(0, 1 << nbits, size=2000, dtype=np.uint64))
    raw = np.concatenate([raw, raw[::17]])           # add duplicates
    mu = np.sort(raw)
    prev = O.keep_mask(mu, nbits, 0)
    assert np.array_equal(prev, np.concatenate([[1], (mu[1:] != mu[:-1]).astype(np.uint8)]))
    for level in range(1, 6):
        cur = O.keep_mask(mu, nbits, level)
        kept_prev = np.nonzero(prev)[0]
        keep = _delta_rule_pass(mu[kept_prev], nbits)
        expect = np.zeros_like(prev)
        expect[kept_prev[np.array(keep, dtype=bool)]] = 1
        assert np.array_equal(cur, expect), level
        assert cur[0] == 1
        assert np.all(cur <= prev)                      # leaves only merge
        prev = cur


@pytest.mark.parametrize("side", [8, 16])
def test_reduction_halves_leaves_on_power_of_two_lattice(side):
    """Closed form: on a side^3 lattice with side = 2^k and jitter well inside a cell, the top 3k
    bits of the 63-bit codes enumerate every lattice cell exactly once, so the radix tree of the
    codes is a perfect binary tree of depth 3k; every pass pairs all leaves with their siblings and
    removes one of each pair, leaving again a perfect tree: the leaf counts are side^3 / 2^level."""
    from paper_2503_09713_gb300 import workloads
    w = workloads.lattice(side, seed=12345)
    mu, _ = O.sort_by_key(O.morton(w["x"], w["y"], w["z"], bits=21))
    counts = [int(O.keep_mask(mu, 63, level).sum()) for level in range(7)]
    assert counts == [side ** 3 >> level for level in range(7)]


def _prefix_box(c1, c2, nbits_axis):
    """Prefix-class box of two 3*b-bit codes (Eqs. lowboundbox, highboundbox), as integer corners."""
    nb = 3 * nbits_axis
    d = O.delta(int(c1), int(c2), nb)
    mask = ((1 << nb) - 1) << (nb - d) & ((1 << nb) - 1)
    p0 = int(c1) & mask
    p1 = p0 + ((1 << (nb - d)) - 1)
    lo = O.deinterleave(p0, nbits_axis)
    hi = O.deinterleave(p1, nbits_axis)
    return np.array(lo), np.array(hi)


def test_cell_boxes_brute_and_prefix_box():
    """Tight cell boxes equal min/max over the cell's particles and lie inside the cell's prefix
    box (App. C 'Compute tree cell sizes')."""
    rng = np.random.default_rng(7)
    n = 3000
    x, y, z = rng.uniform(0, 1, size=(3, n))
    h = rng.uniform(0.01, 0.02, size=n)
    bits = 21
    m = O.morton(x, y, z, bits=bits)
    mu, perm = O.sort_by_key(m)
    xs, ys, zs, hs = x[perm], y[perm], z[perm], h[perm]
    xi = O.keep_mask(mu, 3 * bits, 2)
    idv, ml = O.compact(mu, xi)
    t = O.radix_tree(ml, 3 * bits)
    bmin, bmax, hmax = O.cell_boxes(idv, t.endrange, xs, ys, zs, hs)
    L = len(ml)
    scale = float(1 << bits)
    for c in range(0, 2 * L - 1, 37):
        if c < L - 1:
            lo, hi = min(c, t.endrange[c]), max(c, t.endrange[c])
        else:
            lo = hi = c - (L - 1)
        sl = slice(idv[lo], idv[hi + 1])
        pts = np.stack([xs[sl], ys[sl], zs[sl]], 1)
        assert np.array_equal(bmin[c], pts.min(0)) and np.array_equal(bmax[c], pts.max(0))
        assert hmax[c] == hs[sl].max()
        # prefix box of the cell's first and last code (internal nodes: the node's range ends)
        c1, c2 = mu[idv[lo]], mu[idv[hi + 1] - 1]
        plo, phi = _prefix_box(c1, c2, bits)
        assert np.all(pts.min(0) >= plo / scale) and np.all(pts.max(0) < (phi + 1) / scale)
