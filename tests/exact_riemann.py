"""Exact solution of the Riemann problem for the ideal-gas Euler equations,
by the standard pressure-function Newton iteration for the star pressure
(as in Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
ch. 4).  Used to pin the oracle in the gas limit (G = 0, Sec. 2.1.1)."""
import numpy as np


def _f(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    r = p / pk  # rarefaction
    f = 2.0 * ck / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * ck) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(WL, WR, g):
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _f(p, rl, pl, cl, g)
        fr, dr = _f(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        pn = max(pn, 1e-12 * p)
        if abs(pn - p) <= 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, g)
    fr, _ = _f(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(WL, WR, g, s):
    """Density, velocity, pressure at similarity coordinates s = x/t."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(WL, WR, g)
    out = np.zeros((3, len(s)))
    gm = (g - 1.0) / (g + 1.0)
    for i, S in enumerate(s):
        if S <= us:  # left of contact
            if ps > pl:
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                SL = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[:, i] = (rl, ul, pl) if S < SL else (rs, us, ps)
            else:
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if S < ul - cl:
                    out[:, i] = (rl, ul, pl)
                elif S > us - cs:
                    out[:, i] = (rs, us, ps)
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - S))
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + S)
                    r = rl * (c / cl) ** (2 / (g - 1))
                    out[:, i] = (r, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                SR = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[:, i] = (rr, ur, pr) if S > SR else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if S > ur + cr:
                    out[:, i] = (rr, ur, pr)
                elif S < us + cs:
                    out[:, i] = (rs, us, ps)
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - S))
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + S)
                    r = rr * (c / cr) ** (2 / (g - 1))
                    out[:, i] = (r, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out
