"""The validation references against published values: the star state of Sod's problem (Toro,
Table 4.2, test 1: p* = 0.30313, u* = 0.92745, rho*_L = 0.42632, rho*_R = 0.26557) and the
conservation of mass, momentum and energy by the sampled exact solution."""
import numpy as np

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
