"""Pins of the oracle's kernel family (Sect. 2.1: B-splines M4, M5, M6; Wendland C2, C4, C6):
3-D normalisation, compact support, continuity, derivative, monotonicity, the mean neighbour
numbers the paper quotes, and conservation of the pair forces with every kernel."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_09713_gb300 import workloads as WL

KERNELS = sorted(O.KERNELS.items(), key=lambda kv: kv[1])
HFACT = {"M4": 1.2, "M5": 1.2, "M6": 1.0, "C2": 1.2, "C4": 1.2, "C6": 1.2}


@pytest.mark.parametrize("name,k", KERNELS)
def test_normalisation_by_quadrature(name, k):
    """4 pi C_norm int_0^R f(q) q^2 dq = 1 (Simpson on a fine grid over the support)."""
    R, C = O.kernel_R(k), O.kernel_C(k)
    q = np.linspace(0.0, R, 40001)
    w = np.array([O.kernel_f(k, t) * t * t for t in q])
    dq = q[1] - q[0]
    integ = dq / 3.0 * (w[0] + w[-1] + 4.0 * w[1:-1:2].sum() + 2.0 * w[2:-1:2].sum())
    assert abs(4.0 * math.pi * C * integ - 1.0) < 1e-9


@pytest.mark.parametrize("name,k", KERNELS)
def test_support_continuity_monotonicity(name, k):
    """f vanishes from R on; f and f' are continuous at the piece boundaries; f decreases on
    [0, R) (so h^3 sum_b W is monotone in h and the density root is unique)."""
    R = O.kernel_R(k)
    assert O.kernel_f(k, R) == 0.0 and O.kernel_f(k, R + 0.3) == 0.0 and O.kernel_df(k, R + 0.3) == 0.0
    assert O.kernel_f(k, 0.0) > 0.0 and O.kernel_df(k, 0.0) == 0.0
    for qb in np.arange(0.5, R + 0.25, 0.5):
        e = 1e-9
        assert abs(O.kernel_f(k, qb - e) - O.kernel_f(k, qb + e)) < 1e-6
        assert abs(O.kernel_df(k, qb - e) - O.kernel_df(k, qb + e)) < 1e-6
    q = np.linspace(0.0, R, 2001)
    f = np.array([O.kernel_f(k, t) for t in q])
    assert np.all(np.diff(f) <= 1e-14)


@pytest.mark.parametrize("name,k", KERNELS)
def test_derivative_finite_difference(name, k):
    R = O.kernel_R(k)
    e = 1e-6
    for q in np.linspace(0.05, R - 0.05, 37):
        fd = (O.kernel_f(k, q + e) - O.kernel_f(k, q - e)) / (2 * e)
        assert abs(O.kernel_df(k, q) - fd) < 1e-6 * (1.0 + O.kernel_f(k, 0.0))
    # the scaled forms W, dW/dr and dW/dh follow from f and f'
    h, r = 0.31, 0.37 * O.kernel_R(k) * 0.31
    fd_r = (O.W(r + e * h, h, k) - O.W(r - e * h, h, k)) / (2 * e * h)
    fd_h = (O.W(r, h * (1 + e), k) - O.W(r, h * (1 - e), k)) / (2 * e * h)
    scale = O.W(0.0, h, k) / h
    assert abs(O.F(r, h, k) - fd_r) < 1e-6 * scale
    assert abs(O.dWdh(r, h, k) - fd_h) < 1e-6 * scale


@pytest.mark.parametrize("name,k", [("M4", 0), ("M6", 2)])
def test_mean_neighbour_number(name, k):
    """Uniform random particles at the density root: the mean number of neighbours inside R h is
    close to 4/3 pi (R hfact)^3: about 60 for M4 with hfact 1.2 (57.9), as the paper states, and 113 for
    M6 with hfact 1.0 (Sect. 4)."""
    rng = np.random.default_rng(17)
    n = 6000
    x, y, z = rng.uniform(size=(3, n))
    hf = HFACT[name]
    R = O.kernel_R(k)
    h = O.density_root(x, y, z, hf, 3.0 * hf * n ** (-1.0 / 3.0), kernel=k)
    off, _ = O.neighbours(x, y, z, h, R)   # pairs within R max(h_a, h_b)
    expect = 4.0 / 3.0 * math.pi * (R * hf) ** 3
    mean = np.mean(np.diff(off))
    assert abs(mean / expect - 1.0) < 0.1, (mean, expect)


@pytest.mark.parametrize("name,k", KERNELS)
def test_lattice_density_and_conservation(name, k):
    """Perfect periodic lattice: the density root gives rho -> rho_0 (h/dx -> hfact within the
    lattice-sum error), and on a jittered, moving state the pair forces conserve momentum and
    the semi-discrete energy rate vanishes, for every kernel."""
    hf = HFACT[name]
    s = WL.perfect_lattice(12, hfact=hf)
    h = O.density_root(s["x"], s["y"], s["z"], hf, 2.0 * hf * s["dx"], kernel=k)
    assert np.max(np.abs(h / (hf * s["dx"]) - 1.0)) < 0.02
    assert np.ptp(h) < 1e-12 * h[0]
    w = WL.lattice(10, sigma_v=0.2, jitter=0.15, seed=5 + k, hfact=hf)
    w["u"] = 1.0 + 0.5 * np.random.default_rng(9).uniform(size=w["n"])
    P = O.Params(kernel=k, hfact=hf)
    hh, rho, om, _, _ = O.density_algF(w["x"], w["y"], w["z"], w["h"], w["mass"], P)
    ax, ay, az, du, vs = O.forces(w["x"], w["y"], w["z"], w["vx"], w["vy"], w["vz"], w["u"], hh, om, w["mass"], P)
    m = w["mass"]
    amag = np.abs(np.stack([ax, ay, az])).max()
    assert np.max(np.abs([np.sum(m * ax), np.sum(m * ay), np.sum(m * az)])) < 1e-13 * amag
    e_rate = np.sum(m * (w["vx"] * ax + w["vy"] * ay + w["vz"] * az + du))
    scale = np.sum(m * (np.abs(w["vx"] * ax) + np.abs(w["vy"] * ay) + np.abs(w["vz"] * az) + np.abs(du)))
    assert abs(e_rate) < 1e-12 * scale
