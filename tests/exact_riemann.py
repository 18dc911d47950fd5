"""Exact Riemann solution of the 1D Euler equations for an ideal gas.

Written from the gas dynamics (Rankine-Hugoniot shock curves and isentropic
rarefaction curves, star pressure found by Newton iteration); independent of
the scheme under test.  Used as the closed-form reference for Sod's problem.
"""
import numpy as np


def _wave_curve(p, rho, pk, g):
    """Velocity change across the wave connecting state (rho, pk) to pressure p,
    and its derivative."""
    c = np.sqrt(g * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * c / (g - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * c)


def star_state(L, R, g):
    rl, ul, pl = L
    rr, ur, pr = R
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _wave_curve(p, rl, pl, g)
        fr, dr = _wave_curve(p, rr, pr, g)
        f = fl + fr + ur - ul
        dp = -f / (dl + dr)
        p_new = max(p + dp, 1e-14)
        if abs(p_new - p) < 1e-15 * p:
            p = p_new
            break
        p = p_new
    fl, _ = _wave_curve(p, rl, pl, g)
    fr, _ = _wave_curve(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(L, R, g, xi):
    """Primitive (rho, u, p) at similarity coordinate xi = (x - x0) / t."""
    rl, ul, pl = L
    rr, ur, pr = R
    ps, us = star_state(L, R, g)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            r, u, p, sign = rl, ul, pl, -1.0
        else:
            r, u, p, sign = rr, ur, pr, 1.0
        c = np.sqrt(g * p / r)
        if ps > p:  # shock
            rs = r * ((ps / p + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / p + 1))
            S = u + sign * c * np.sqrt((g + 1) / (2 * g) * ps / p + (g - 1) / (2 * g))
            if sign * (s - S) >= 0:
                out[:, n] = (r, u, p)
            else:
                out[:, n] = (rs, us, ps)
        else:  # rarefaction
            rs = r * (ps / p) ** (1.0 / g)
            cs = c * (ps / p) ** ((g - 1) / (2 * g))
            head = u + sign * c
            tail = us + sign * cs
            if sign * (s - head) >= 0:
                out[:, n] = (r, u, p)
            elif sign * (s - tail) <= 0:
                out[:, n] = (rs, us, ps)
            else:
                uu = 2.0 / (g + 1) * (-sign * c + (g - 1) / 2 * u + s)
                cc = 2.0 / (g + 1) * c - sign * (g - 1) / (g + 1) * (u - s)
                rr_ = r * (cc / c) ** (2.0 / (g - 1))
                pp = p * (cc / c) ** (2.0 * g / (g - 1))
                out[:, n] = (rr_, uu, pp)
    return out
