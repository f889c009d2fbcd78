"""Closed-form references for the validation runs (Sect. 4 of the paper: Sod tube, Sedov-Taylor blast).

* Exact solution of the Riemann problem of gas dynamics (Sod 1978; the construction of Toro,
  "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4): star pressure from
  f_L(p) + f_R(p) + u_R - u_L = 0 with the shock / rarefaction branches of f_K, then sampling of the
  self-similar wave pattern at S = (x - x0)/t.
* Sedov-Taylor blast: shock radius R(t) = xi_0 (E t^2 / rho_0)^(1/5), xi_0 = 1.15167 for gamma = 5/3
  in 3-D (Sedov 1959), and the strong-shock density jump (gamma + 1)/(gamma - 1).  The profiles
  behind the shock come from the classical closed-form similarity solution of the strong point
  explosion (Sedov 1959; Landau & Lifshitz, Fluid Mechanics, the section on the strong explosion),
  written in the velocity variable V of v = (2 r / 5 t) V, which runs from 2/(gamma+1) at the shock to
  1/gamma at the centre; xi_0 follows from the energy integral of those profiles.
Plain numpy, used by tests only.
"""
import math

import numpy as np

SEDOV_XI0_GAMMA_5_3 = 1.15167


def _fk(p, rho, pk, ck, g):
    """Toro's pressure function of one side and its derivative."""
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))   # rarefaction
    return 2.0 * ck / (g - 1.0) * (r - 1.0), 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def riemann_star(left, right, g):
    """(p*, u*) of the Riemann problem with states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, cl, g)
        fr, dr = _fk(p, rr, pr, cr, g)
        pn = max(1e-14, p - (fl + fr + ur - ul) / (dl + dr))
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def riemann_sample(x, t, x0, left, right, g):
    """(rho, u, p) of the exact solution at positions x (array) and time t > 0."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = riemann_star(left, right, g)
    S = (np.asarray(x, dtype=float) - x0) / t
    rho, u, p = np.empty_like(S), np.empty_like(S), np.empty_like(S)
    gm = (g - 1.0) / (g + 1.0)
    for i, s in enumerate(S):
        if s <= us:   # left of the contact
            if ps > pl:   # left shock
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= sl:
                    rho[i], u[i], p[i] = rl, ul, pl
                else:
                    rho[i], u[i], p[i] = rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
            else:   # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                if s <= ul - cl:
                    rho[i], u[i], p[i] = rl, ul, pl
                elif s >= us - csl:
                    rho[i], u[i], p[i] = rl * (ps / pl) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    u[i] = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    rho[i] = rl * (c / cl) ** (2.0 / (g - 1.0))
                    p[i] = pl * (c / cl) ** (2.0 * g / (g - 1.0))
        else:   # right of the contact
            if ps > pr:   # right shock
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= sr:
                    rho[i], u[i], p[i] = rr, ur, pr
                else:
                    rho[i], u[i], p[i] = rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
            else:   # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                if s >= ur + cr:
                    rho[i], u[i], p[i] = rr, ur, pr
                elif s <= us + csr:
                    rho[i], u[i], p[i] = rr * (ps / pr) ** (1.0 / g), us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    u[i] = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    rho[i] = rr * (c / cr) ** (2.0 / (g - 1.0))
                    p[i] = pr * (c / cr) ** (2.0 * g / (g - 1.0))
    return rho, u, p


def sedov_radius(t, energy=1.0, rho0=1.0, xi0=SEDOV_XI0_GAMMA_5_3):
    return xi0 * (energy * t * t / rho0) ** 0.2


# ------------------------------------------------------------------------------ Sedov-Taylor profiles
def _sedov_exponents(g):
    n1 = -(13.0 * g * g - 7.0 * g + 12.0) / ((3.0 * g - 1.0) * (2.0 * g + 1.0))
    n2 = 5.0 * (g - 1.0) / (2.0 * g + 1.0)
    n3 = 3.0 / (2.0 * g + 1.0)
    n4 = -n1 / (2.0 - g)
    n5 = -2.0 / (2.0 - g)
    return n1, n2, n3, n4, n5


def sedov_similarity(V, g):
    """(lambda = r/R, G = rho/rho_0, Z) of the spherical strong explosion as functions of V, with
    v = (2 r / 5 t) V, rho = rho_0 G and c^2 = gamma P / rho = (2 r / 5 t)^2 Z.  Each bracket below
    equals 1 at the shock (V = 2/(gamma+1)); gamma V - 1 vanishes at the centre (V = 1/gamma)."""
    V = np.asarray(V, dtype=float)
    n1, n2, n3, n4, n5 = _sedov_exponents(g)
    b1 = 0.5 * (g + 1.0) * V
    b2 = (g + 1.0) / (7.0 - g) * (5.0 - (3.0 * g - 1.0) * V)
    b3 = (g + 1.0) / (g - 1.0) * (g * V - 1.0)
    b4 = (g + 1.0) / (g - 1.0) * (1.0 - V)
    lam = (b1 ** -2.0 * b2 ** n1 * b3 ** n2) ** 0.2
    G = (g + 1.0) / (g - 1.0) * b3 ** n3 * b2 ** n4 * b4 ** n5
    Z = g * (g - 1.0) * (1.0 - V) * V * V / (2.0 * (g * V - 1.0))
    return lam, G, Z


def _sedov_table(g, n=20001):
    """The similarity functions on a V grid clustered towards the centre (lambda ~ (gamma V - 1)^(n2/5))."""
    v_s, v_c = 2.0 / (g + 1.0), 1.0 / g
    u = np.linspace(0.0, 1.0, n)
    V = v_c + (v_s - v_c) * u ** 3          # u = 0: centre, u = 1: shock
    V[0] = v_c * (1.0 + 1e-15)
    with np.errstate(divide="ignore"):
        lam, G, Z = sedov_similarity(V, g)
    lam[0], G[0], Z[0] = 0.0, 0.0, Z[1]   # centre: G -> 0 while G Z lambda^2 (the pressure) stays finite
    return V, lam, G, Z


def sedov_integrals(g):
    """(int_0^1 G lambda^2 dlambda, int_0^1 G lambda^4 (V^2/2 + Z/(gamma (gamma-1))) dlambda): the
    first is 1/3 by mass conservation (the swept-up mass), the second fixes xi_0 through
    E = (16 pi / 25) xi_0^5 E I."""
    V, lam, G, Z = _sedov_table(g)
    mass = np.trapezoid(G * lam ** 2, lam)
    energy = np.trapezoid(G * lam ** 4 * (0.5 * V * V + Z / (g * (g - 1.0))), lam)
    return mass, energy


def sedov_xi0(g):
    """xi_0 of R = xi_0 (E t^2 / rho_0)^(1/5) from the energy integral of the profiles."""
    _, I = sedov_integrals(g)
    return (25.0 / (16.0 * math.pi * I)) ** 0.2


def sedov_profile(r, t, g, energy=1.0, rho0=1.0):
    """(rho, v_r, P) of the exact blast at radii r (array) and time t; ambient state (rho0, 0, 0)
    outside the shock."""
    xi0 = sedov_xi0(g)
    R = xi0 * (energy * t * t / rho0) ** 0.2
    V, lam, G, Z = _sedov_table(g)
    r = np.asarray(r, dtype=float)
    lam_r = np.clip(r / R, 0.0, None)
    inside = lam_r < 1.0
    Vi = np.interp(lam_r, lam, V)
    Gi = np.interp(lam_r, lam, G)
    Zi = np.interp(lam_r, lam, Z)
    w = 2.0 * r / (5.0 * t)
    rho = np.where(inside, rho0 * Gi, rho0)
    v = np.where(inside, w * Vi, 0.0)
    P = np.where(inside, rho0 * Gi * w * w * Zi / g, 0.0)
    return rho, v, P
