"""Exact reference solutions used to pin the oracle (test infrastructure).

* ``riemann_euler``: exact solution of the Riemann problem of the 1-D Euler
  equations for an ideal gas, written from the published method of Toro,
  "Riemann Solvers and Numerical Methods for Fluid Dynamics", Ch. 4 (the book
  the paper cites for its spherical Sod test, Sec. 4 "Spherical Riemann
  problem"): Newton iteration for the star pressure on
  f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0 and self-similar sampling.
* ``shift_periodic``: exact translation of a periodic profile (smooth
  advection and circularly polarised Alfven waves, Sec. 4 "Circularly
  polarised Alfven waves": the profile returns to its initial state after
  one period).
"""
from __future__ import annotations

import math

import numpy as np


def _f_side(p, rho, pk, gamma):
    """Pressure function f_K(p) and its derivative for one side (shock if p > p_K,
    rarefaction otherwise)."""
    ck = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        f = (p - pk) * q
        df = q * (1.0 - 0.5 * (p - pk) / (B + p))
    else:
        pr = p / pk
        f = 2.0 * ck / (gamma - 1.0) * (pr ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
        df = 1.0 / (rho * ck) * pr ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma, tol=1e-14, maxit=200):
    """Star-region pressure and velocity (p*, u*) of the Riemann problem
    ``left = (rho, u, p)``, ``right = (rho, u, p)``."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    if 2.0 / (gamma - 1.0) * (cl + cr) <= ur - ul:
        raise ValueError("vacuum is generated; not handled")
    # two-rarefaction initial guess
    z = (gamma - 1.0) / (2.0 * gamma)
    p = ((cl + cr - 0.5 * (gamma - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(maxit):
        fl, dfl = _f_side(p, rl, pl, gamma)
        fr, dfr = _f_side(p, rr, pr, gamma)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) / (0.5 * (pn + p)) < tol:
            p = pn
            break
        p = pn
    fl, _ = _f_side(p, rl, pl, gamma)
    fr, _ = _f_side(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_euler(left, right, gamma, xi):
    """Sample the exact solution at similarity coordinates ``xi = (x - x0)/t``.
    Returns arrays (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    g = gamma
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for n, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    r, v, q = rl, ul, pl
                else:
                    r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                    v, q = us, ps
            else:  # left rarefaction
                shl = ul - cl
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - csl
                if s <= shl:
                    r, v, q = rl, ul, pl
                elif s >= stl:
                    r = rl * (ps / pl) ** (1 / g)
                    v, q = us, ps
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    v = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    r = rl * (c / cl) ** (2 / (g - 1))
                    q = pl * (c / cl) ** (2 * g / (g - 1))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    r, v, q = rr, ur, pr
                else:
                    r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                    v, q = us, ps
            else:  # right rarefaction
                shr = ur + cr
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + csr
                if s >= shr:
                    r, v, q = rr, ur, pr
                elif s <= str_:
                    r = rr * (ps / pr) ** (1 / g)
                    v, q = us, ps
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    v = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    r = rr * (c / cr) ** (2 / (g - 1))
                    q = pr * (c / cr) ** (2 * g / (g - 1))
        rho[n], u[n], p[n] = r, v, q
    return rho, u, p


def riemann_cell_averages(left, right, gamma, x_faces, x0, t, sub=64):
    """Cell averages of the exact Riemann density/velocity/pressure over cells
    bounded by ``x_faces`` (midpoint rule with ``sub`` points per cell)."""
    xf = np.asarray(x_faces, dtype=np.float64)
    n = xf.size - 1
    frac = (np.arange(sub) + 0.5) / sub
    pts = xf[:-1, None] + (xf[1:] - xf[:-1])[:, None] * frac[None, :]
    r, u, p = riemann_euler(left, right, gamma, (pts.ravel() - x0) / t)
    return (r.reshape(n, sub).mean(1), u.reshape(n, sub).mean(1), p.reshape(n, sub).mean(1))


def shift_periodic(profile_fn, x, shift):
    """Exact translation of a periodic profile: profile(x - shift)."""
    return profile_fn(np.asarray(x) - shift)
