"""Steady one-dimensional C-shock structure from the conservation laws and
the non-ideal induction law, for checking the oracle's Ohmic and ambipolar
terms (DISPATCH I, Sec. 4.3, validated in Sec. 5.4 against Table 1).

In a frame where the shock is at rest and everything depends on x alone,
the fluxes of mass, x- and y-momentum, energy and B_y are constant through
the shock.  With E_z = -(v_x B_y - v_y B_x) + E_ni, constant E_z gives the
non-ideal field E_ni = E_z0 + v_x B_y - v_y B_x, and the non-ideal law
relates it to the current J_z = dB_y/dx:
    Ohmic (Eq. 2):       E_ni = eta J_z
    ambipolar (Eqs. 5-6): E_ni = |B|^2 J_z / (gamma_AD rho rho_i)   (B.J = 0)
Given B_y, the other variables follow algebraically from the constant
fluxes (the energy flux includes the Poynting flux -E_ni B_y of the
non-ideal field; the isothermal case uses p = c_s^2 rho instead), so the
structure is an ODE for B_y(x), integrated from the upstream state.
Heaviside-Lorentz units (magnetic pressure B^2/2).
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cshock_table1.txt")


def table1():
    """Rows of Table 1 as {name: (rho, vx, vy, Bx, By, P)}."""
    env = {"sqrt": np.sqrt}
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if not line:
            continue
        rows[line[0]] = tuple(float(eval(v, env)) for v in line[1:])
    return rows


def fluxes(state, gamma):
    """Ideal-MHD x-fluxes of mass, x- and y-momentum and energy, and the
    B_y flux v_x B_y - v_y B_x, of a state (rho, vx, vy, Bx, By, P) with
    v_z = B_z = 0."""
    rho, vx, vy, Bx, By, p = state
    B2 = Bx * Bx + By * By
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy) + 0.5 * B2
    PT = p + 0.5 * B2
    return np.array([rho * vx, rho * vx * vx + PT - Bx * Bx, rho * vx * vy - Bx * By,
                     (E + PT) * vx - Bx * (vx * Bx + vy * By), vx * By - vy * Bx])


class CShock:
    """The steady structure from upstream state `pre`; law 'ohm' (coef =
    eta) or 'ad' (coef = gamma_AD); isothermal: p / rho fixed."""

    def __init__(self, pre, gamma, law, coef, rho_i=1.0, isothermal=False):
        self.pre = pre
        rho0, vx0, vy0, Bx, By0, p0 = pre
        self.j = rho0 * vx0
        self.Pi = self.j * vx0 + p0 + 0.5 * By0 ** 2
        self.Cy = self.j * vy0 - Bx * By0
        self.Ez0 = -(vx0 * By0 - vy0 * Bx)
        self.g1 = gamma / (gamma - 1.0)
        self.FE0 = (0.5 * rho0 * (vx0 ** 2 + vy0 ** 2) + self.g1 * p0 + Bx ** 2 + By0 ** 2) * vx0 \
            - Bx * (vx0 * Bx + vy0 * By0)
        self.cs2 = p0 / rho0
        self.Bx, self.law, self.coef, self.rho_i, self.iso = Bx, law, coef, rho_i, isothermal

    def state(self, By):
        """(rho, vx, vy, p, E_ni) on the supersonic branch for a given B_y."""
        j, Bx = self.j, self.Bx
        vy = (self.Cy + Bx * By) / j
        if self.iso:
            A = self.Pi - 0.5 * By ** 2
            rho = (A - np.sqrt(A * A - 4.0 * self.cs2 * j * j)) / (2.0 * self.cs2)
            vx = j / rho
            p = self.cs2 * rho
        else:
            a = j * (0.5 - self.g1)
            b = self.g1 * (self.Pi - 0.5 * By ** 2)
            c = 0.5 * j * vy ** 2 - self.Ez0 * By - self.FE0
            vx = (-b - np.sqrt(b * b - 4.0 * a * c)) / (2.0 * a)
            rho = j / vx
            p = self.Pi - j * vx - 0.5 * By ** 2
        Eni = self.Ez0 + vx * By - vy * Bx
        return rho, vx, vy, p, Eni

    def rhs(self, x, y):
        By = y[0]
        rho, vx, vy, p, Eni = self.state(By)
        if self.law == "ohm":
            return [Eni / self.coef]
        return [self.coef * rho * self.rho_i * Eni / (self.Bx * self.Bx + By * By)]

    def solve(self, length=6.0):
        """Integrate B_y from just above the upstream value; returns the
        dense solution (x from 0)."""
        from scipy.integrate import solve_ivp
        return solve_ivp(self.rhs, (0.0, length), [self.pre[4] * (1.0 + 1e-8)], rtol=1e-12, atol=1e-14,
                         dense_output=True, max_step=0.005)


# The three experiments of Sec. 5.4: Table 1 rows, gamma, law and coefficient
# (gamma_AD = 75, eta = 0.1, rho_i = 1), isothermal or not.
CASES = {
    "ad_iso": ("ad_pre", "ad_iso_post", 1.0 + 1e-7, "ad", 75.0, True),
    "ad_noniso": ("ad_pre", "ad_noniso_post", 5.0 / 3.0, "ad", 75.0, False),
    "ohm": ("ohm_pre", "ohm_post", 5.0 / 3.0, "ohm", 0.1, False),
}


def law_kw(law, coef):
    """Keyword arguments of the non-ideal term of a case."""
    return dict(eta=coef) if law == "ohm" else dict(gamma_ad=coef, rho_i=1.0)


def jump_input(name, ncell=300, Lx=4.0, xs=3.0):
    """Sec. 5.4's initial condition: the Table 1 pre-shock state for x < xs,
    the post-shock state beyond, on a periodic box of length Lx cut into
    patches of 30 x 4 x 4 cells (dx = Lx / ncell).  Returns the layout, the
    fields, gamma, the non-ideal keyword arguments and the cell centres."""
    from paper_1705_10774_gb300 import ics
    rows = table1()
    pre_n, post_n, gamma, law, coef, iso = CASES[name]
    pre, post = rows[pre_n], rows[post_n]
    dx = Lx / ncell
    lay = ics.cartesian((ncell // 30, 1, 1), (30, 4, 4), dx=dx)
    X, Y, Z = lay.base_cells
    xc = (np.arange(X) + 0.5) * dx
    up = xc < xs
    shape = (Z, Y, X)
    bc = lambda a: np.broadcast_to(a, shape).copy()
    sel = lambda k: np.where(up, pre[k], post[k])
    f = ics.Fields(rho=bc(sel(0)), v=np.stack([bc(sel(1)), bc(sel(2)), bc(0 * xc)]), p=bc(sel(5)),
                   bx=bc(0 * xc + pre[3]), by=bc(sel(4)), bz=bc(0 * xc), gamma=gamma)
    return lay, f, gamma, law_kw(law, coef), xc


def profile_error(name, xc, By, xs):
    """Mean |B_y - steady profile| within 0.3 of the shock over the jump in
    B_y, the steady profile aligned with B_y at its mid-value crossing near
    xs."""
    rows = table1()
    pre_n, post_n, gamma, law, coef, iso = CASES[name]
    pre, post = rows[pre_n], rows[post_n]
    sol = CShock(pre, gamma, law, coef, isothermal=iso).solve()
    mid = 0.5 * (pre[4] + post[4])
    dx = xc[1] - xc[0]
    i = np.where((np.abs(xc - xs) < 0.6) & (By > mid))[0][0]
    xcross = xc[i - 1] + (mid - By[i - 1]) / (By[i] - By[i - 1]) * dx
    s = xc - xcross + sol.t[np.argmax(sol.y[0] > mid)]
    ode = np.where(s <= 0, pre[4], sol.sol(np.clip(s, 0, sol.t[-1]))[0])
    w = np.abs(xc - xcross) < 0.3
    return float(np.abs(By - ode)[w].mean() / abs(post[4] - pre[4]))


def most_common_steps(schedule, npatch):
    """Each patch's most frequent step in a schedule (patch, t, dt)."""
    sp, _, sd = schedule
    out = []
    for P in range(npatch):
        vals, cnt = np.unique(sd[sp == P], return_counts=True)
        out.append(vals[np.argmax(cnt)])
    return np.array(out)
