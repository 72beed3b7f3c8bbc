"""Exact solution of the 1D Euler Riemann problem for an ideal gas, written
from the standard textbook construction (Toro, "Riemann Solvers and Numerical
Methods for Fluid Dynamics", Ch. 4): Newton iteration for the star pressure
on f_L(p) + f_R(p) + (u_R - u_L) = 0, then sampling of the self-similar
solution.  Used to pin the oracle's B = 0 (hydro) limit on the Sod problem."""
import math

import numpy as np


def _fk(p, rho, pk, gam):
    a = math.sqrt(gam * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gam + 1.0) * rho)
        B = (gam - 1.0) / (gam + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    r = (p / pk) ** ((gam - 1.0) / (2.0 * gam))
    f = 2.0 * a / (gam - 1.0) * (r - 1.0)
    df = 1.0 / (rho * a) * (p / pk) ** (-(gam + 1.0) / (2.0 * gam))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, gam):
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, gam)
        fr, dfr = _fk(p, rr, pr, gam)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(p - dp, 1e-12)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, gam)
    fr, _ = _fk(p, rr, pr, gam)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    def rho_star(rk, pk):
        if p > pk:
            g = (gam - 1.0) / (gam + 1.0)
            return rk * (p / pk + g) / (g * p / pk + 1.0)
        return rk * (p / pk) ** (1.0 / gam)
    return p, u, rho_star(rl, pl), rho_star(rr, pr)


def sample(x, t, x0, rl, ul, pl, rr, ur, pr, gam):
    """Density, velocity, pressure at positions x at time t."""
    ps, us, rsl, rsr = star_state(rl, ul, pl, rr, ur, pr, gam)
    al, ar = math.sqrt(gam * pl / rl), math.sqrt(gam * pr / rr)
    out = np.zeros((3, len(x)))
    for i, xi in enumerate(x):
        s = (xi - x0) / t
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - al * math.sqrt((gam + 1) / (2 * gam) * ps / pl + (gam - 1) / (2 * gam))
                out[:, i] = (rl, ul, pl) if s < sl else (rsl, us, ps)
            else:
                shl = ul - al
                astar = al * (ps / pl) ** ((gam - 1) / (2 * gam))
                stl = us - astar
                if s < shl:
                    out[:, i] = (rl, ul, pl)
                elif s > stl:
                    out[:, i] = (rsl, us, ps)
                else:
                    u = 2 / (gam + 1) * (al + (gam - 1) / 2 * ul + s)
                    c = 2 / (gam + 1) * (al + (gam - 1) / 2 * (ul - s))
                    r = rl * (c / al) ** (2 / (gam - 1))
                    out[:, i] = (r, u, pl * (c / al) ** (2 * gam / (gam - 1)))
        else:
            if ps > pr:
                sr = ur + ar * math.sqrt((gam + 1) / (2 * gam) * ps / pr + (gam - 1) / (2 * gam))
                out[:, i] = (rr, ur, pr) if s > sr else (rsr, us, ps)
            else:
                shr = ur + ar
                astar = ar * (ps / pr) ** ((gam - 1) / (2 * gam))
                str_ = us + astar
                if s > shr:
                    out[:, i] = (rr, ur, pr)
                elif s < str_:
                    out[:, i] = (rsr, us, ps)
                else:
                    u = 2 / (gam + 1) * (-ar + (gam - 1) / 2 * ur + s)
                    c = 2 / (gam + 1) * (ar - (gam - 1) / 2 * (ur - s))
                    r = rr * (c / ar) ** (2 / (gam - 1))
                    out[:, i] = (r, u, pr * (c / ar) ** (2 * gam / (gam - 1)))
    return out
