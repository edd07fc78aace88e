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
