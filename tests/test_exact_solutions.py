"""The validation references against published values: the star state of Sod's problem (Toro,
Table 4.2, test 1: p* = 0.30313, u* = 0.92745, rho*_L = 0.42632, rho*_R = 0.26557) and the
conservation of mass, momentum and energy by the sampled exact solution; the Sedov-Taylor
similarity solution against the strong-shock jump, mass conservation, its energy integral and the
published values of xi_0."""
import math

import numpy as np
import pytest

import exact_solutions as E
from exact_solutions import riemann_sample, riemann_star

SOD_L, SOD_R, G = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4


def test_sod_star_state():
    ps, us = riemann_star(SOD_L, SOD_R, G)
    assert abs(ps - 0.30313) < 5e-6 and abs(us - 0.92745) < 5e-6
    rho, u, p = riemann_sample(np.array([0.5 + 0.2 * us - 1e-9, 0.5 + 0.2 * us + 1e-9]), 0.2, 0.5,
                               SOD_L, SOD_R, G)
    assert abs(rho[0] - 0.42632) < 5e-5 and abs(rho[1] - 0.26557) < 5e-5


def test_exact_solution_conserves():
    """Over a domain the waves have not left, the integrals of rho and E = p/(gamma-1) + rho u^2/2
    do not change (no flux at ends at rest) and the momentum integral grows by the pressure
    difference of the ends times t."""
    x = np.linspace(-0.5, 1.5, 200001)
    dx = x[1] - x[0]
    t = 0.245
    r0, u0, p0 = riemann_sample(x, 1e-9, 0.5, SOD_L, SOD_R, G)
    r1, u1, p1 = riemann_sample(x, t, 0.5, SOD_L, SOD_R, G)
    assert abs(np.sum(r1 - r0) * dx) < 2e-5
    e0 = p0 / (G - 1) + 0.5 * r0 * u0 ** 2
    e1 = p1 / (G - 1) + 0.5 * r1 * u1 ** 2
    assert abs(np.sum(e1 - e0) * dx) < 5e-5
    assert abs(np.sum(r1 * u1 - r0 * u0) * dx - (SOD_L[2] - SOD_R[2]) * t) < 5e-5


@pytest.mark.parametrize("g", [5.0 / 3.0, 1.4])
def test_sedov_similarity_shock_state(g):
    """At the shock (V = 2/(gamma+1)) the similarity functions give the strong-shock
    (Rankine-Hugoniot) state: r = R, rho = rho_0 (gamma+1)/(gamma-1), and c^2 = 2 gamma (gamma-1)
    Rdot^2/(gamma+1)^2, i.e. P = 2 rho_0 Rdot^2/(gamma+1), v = 2 Rdot/(gamma+1)."""
    lam, G, Z = E.sedov_similarity(np.array([2.0 / (g + 1.0)]), g)
    assert lam[0] == pytest.approx(1.0, rel=1e-14)
    assert G[0] == pytest.approx((g + 1.0) / (g - 1.0), rel=1e-14)
    assert Z[0] == pytest.approx(2.0 * g * (g - 1.0) / (g + 1.0) ** 2, rel=1e-14)


@pytest.mark.parametrize("g", [5.0 / 3.0, 1.4])
def test_sedov_similarity_mass_integral(g):
    """The blast sweeps up the ambient mass: int_0^1 G lambda^2 dlambda = 1/3."""
    mass, _ = E.sedov_integrals(g)
    assert mass == pytest.approx(1.0 / 3.0, rel=1e-6)


def test_sedov_xi0_published_values():
    """xi_0 from the energy integral of the profiles: 1.15167 for gamma = 5/3 (the constant the
    paper's comparison uses) and 1.033 for gamma = 1.4 (Sedov's value for air)."""
    assert E.sedov_xi0(5.0 / 3.0) == pytest.approx(E.SEDOV_XI0_GAMMA_5_3, abs=2e-5)
    assert E.sedov_xi0(1.4) == pytest.approx(1.033, abs=1e-3)


def test_sedov_profile_energy_and_mass():
    """The sampled profile at t holds the blast energy E and the swept mass: int (rho v^2/2 +
    P/(gamma-1)) 4 pi r^2 dr = E and int rho 4 pi r^2 dr = 4/3 pi R^3 rho_0 (checks the v and P
    scalings of sedov_profile, not only the similarity functions)."""
    g, t, energy = 5.0 / 3.0, 0.05, 1.0
    R = E.sedov_radius(t, energy)
    r = np.linspace(0.0, R * (1 - 1e-9), 400001)
    rho, v, P = E.sedov_profile(r, t, g, energy)
    e = np.trapezoid((0.5 * rho * v * v + P / (g - 1.0)) * 4.0 * math.pi * r * r, r)
    m = np.trapezoid(rho * 4.0 * math.pi * r * r, r)
    assert e == pytest.approx(energy, rel=2e-3)
    assert m == pytest.approx(4.0 / 3.0 * math.pi * R ** 3, rel=2e-3)
