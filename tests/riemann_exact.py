"""Exact solution of the Riemann problem of the 1-D Euler equations for an
ideal gas, written from the mathematics (Godunov's pressure function, solved
for the star pressure by Newton iteration; see Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4).  Used as an independent pin of
the oracle's shock-tube results."""
import numpy as np


def _fk(p, rho, pk, gamma):
    """Velocity jump across the wave that connects state k to pressure p, and
    its derivative."""
    a = np.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    r = (p / pk) ** ((gamma - 1.0) / (2.0 * gamma))
    f = 2.0 * a / (gamma - 1.0) * (r - 1.0)
    df = 1.0 / (rho * a) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, gamma):
    """Star-region pressure and velocity."""
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, gamma)
        fr, dr = _fk(p, rr, pr, gamma)
        f = fl + fr + (ur - ul)
        pn = p - f / (dl + dr)
        if pn <= 0:
            pn = 1e-8 * p
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, gamma)
    fr, _ = _fk(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, rl, ul, pl, rr, ur, pr, gamma):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    ps, us = star_state(rl, ul, pl, rr, ur, pr, gamma)
    g = gamma
    out = np.zeros((3,) + np.shape(xi))
    xi = np.asarray(xi, float)
    al = np.sqrt(g * pl / rl)
    ar = np.sqrt(g * pr / rr)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:
                SL = ul - al * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= SL:
                    val = (rl, ul, pl)
                else:
                    r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                    val = (r, us, ps)
            else:
                SHL = ul - al
                ast = al * (ps / pl) ** ((g - 1) / (2 * g))
                STL = us - ast
                if s <= SHL:
                    val = (rl, ul, pl)
                elif s >= STL:
                    val = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
                    val = (rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + s),
                           pl * c ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                SR = ur + ar * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= SR:
                    val = (rr, ur, pr)
                else:
                    r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                    val = (r, us, ps)
            else:
                SHR = ur + ar
                ast = ar * (ps / pr) ** ((g - 1) / (2 * g))
                STR = us + ast
                if s >= SHR:
                    val = (rr, ur, pr)
                elif s <= STR:
                    val = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
                    val = (rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s),
                           pr * c ** (2 * g / (g - 1)))
        out[(slice(None),) + idx] = val
    return out
