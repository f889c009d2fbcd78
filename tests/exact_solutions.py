"""Closed-form references for the validation runs (Sect. 4 of the paper: Sod tube, Sedov-Taylor blast).

* Exact solution of the Riemann problem of gas dynamics (Sod 1978; the construction of Toro,
  "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4): star pressure from
  f_L(p) + f_R(p) + u_R - u_L = 0 with the shock / rarefaction branches of f_K, then sampling of the
  self-similar wave pattern at S = (x - x0)/t.
* Sedov-Taylor blast: shock radius R(t) = xi_0 (E t^2 / rho_0)^(1/5), xi_0 = 1.15167 for gamma = 5/3
  in 3-D (Sedov 1959), and the strong-shock density jump (gamma + 1)/(gamma - 1).
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
