"""Pins of the oracle's HLLD flux (Miyoshi & Kusano 2005; the MHD solver
whose cost Sec. 5.3 compares with RAMSES), each on a property the method is
built to have rather than on the oracle itself: with equal states it is the
physical flux (pinned for HLL by the eigenmode jumps); it resolves an
isolated contact and an isolated rotational (Alfven) discontinuity exactly,
so the flux at the interface is the flux of the exact state there; without
a magnetic field it is the textbook HLLC flux (the hydrodynamic solver Sec.
4.1 ports from RAMSES); it is mirror symmetric; and the full update with it
converges at second order on linear waves, keeps a stationary contact
steady where HLL smears it, and solves the Sod tube no worse than HLL."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1705_10774_gb300 import ics
import riemann_exact as RX
from test_oracle_pins import cons, run

G53 = 5.0 / 3.0


def phys_flux(W, d, g):
    """Physical flux of W along axis d, as HLL and HLLD return it for equal
    states (HLL's version is pinned by the eigenmode-jump test)."""
    return O.hll(W, W, d, g)[0]


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlld_of_equal_states_is_the_physical_flux(d):
    rng = np.random.default_rng(d)
    for _ in range(20):
        W = np.array([0.5 + rng.random(), *(rng.standard_normal(3)), 0.3 + rng.random(),
                      *(rng.standard_normal(3))])
        F, S = O.hlld(W, W, d, G53)
        Fh, Sh = O.hll(W, W, d, G53)
        assert np.allclose(F, Fh, rtol=1e-13, atol=1e-14)
        assert np.array_equal(S, Sh)


def _with(d, rho, u, v, w, p, bn, bt1, bt2):
    """Primitive state with normal axis d given in the normal frame."""
    W = np.zeros(8)
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    W[0] = rho
    W[1 + d], W[1 + t1], W[1 + t2] = u, v, w
    W[4] = p
    W[5 + d], W[5 + t1], W[5 + t2] = bn, bt1, bt2
    return W


@pytest.mark.parametrize("d", [0, 2])
@pytest.mark.parametrize("u", [0.4, 0.0, -0.3])
@pytest.mark.parametrize("bn", [0.0, 0.8])
def test_hlld_resolves_an_isolated_contact(d, u, bn):
    """A jump in density alone (same velocity, pressure and field) is a
    contact moving at u: the exact flux at the interface is the upwind
    state's (both sides agree for u = 0).  HLLD returns it; HLL does not."""
    WL = _with(d, 1.0, u, 0.2, -0.1, 0.7, bn, 0.5, -0.3)
    WR = _with(d, 0.25, u, 0.2, -0.1, 0.7, bn, 0.5, -0.3)
    F, _ = O.hlld(WL, WR, d, G53)
    up = WL if u >= 0 else WR
    Fex = phys_flux(up, d, G53)
    scale = np.max(np.abs(Fex)) + 1.0
    assert np.max(np.abs(F - Fex)) <= 1e-13 * scale
    Fh, _ = O.hll(WL, WR, d, G53)
    assert np.max(np.abs(Fh - Fex)) > 1e-3        # HLL smears the contact


@pytest.mark.parametrize("family", [-1, 1])
@pytest.mark.parametrize("bn", [1.0, -0.7])
@pytest.mark.parametrize("u", [0.3, -0.4, -1.6])
def test_hlld_resolves_an_isolated_rotational_discontinuity(family, bn, u):
    """Rotating the tangential field by a finite angle at fixed |B_t|, with
    the tangential velocity jumping by -family * sign(Bn) dB_t / sqrt(rho),
    is an exact rotational discontinuity moving at u + family |Bn|/sqrt(rho).
    The flux at the interface is the flux of the state on the side the
    discontinuity is moving away from."""
    d = 1
    rho, p = 1.3, 0.8
    bt = np.array([0.6, -0.4])
    th = 1.1
    rot = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    btR = rot @ bt
    vt = np.array([0.25, -0.1])
    vtR = vt - family * np.sign(bn) * (btR - bt) / np.sqrt(rho)
    WL = _with(d, rho, u, vt[0], vt[1], p, bn, bt[0], bt[1])
    WR = _with(d, rho, u, vtR[0], vtR[1], p, bn, btR[0], btR[1])
    lam = u + family * abs(bn) / np.sqrt(rho)
    F, _ = O.hlld(WL, WR, d, G53)
    Fex = phys_flux(WL if lam > 0 else WR, d, G53)
    assert np.max(np.abs(F - Fex)) <= 1e-12 * (np.max(np.abs(Fex)) + 1.0), (lam, F - Fex)
    # the constructed states are a discontinuity moving at lam: the jump of
    # the physical flux is lam times the jump of the conserved variables
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    cU = lambda W: (lambda U: np.concatenate([U[:5], [U[5 + t1], U[5 + t2]]]))(cons(W, G53))
    dF = phys_flux(WR, d, G53) - phys_flux(WL, d, G53)
    assert np.allclose(dF, lam * (cU(WR) - cU(WL)), rtol=1e-12, atol=1e-13)


def test_hlld_mirror_symmetry():
    g = 1.4
    WL = np.array([1.0, 0.2, 0.1, 0.0, 1.0, 0.5, 0.1, 0.3])
    WR = np.array([0.5, -0.3, 0.0, 0.1, 0.4, 0.5, -0.2, 0.1])
    F1, S1 = O.hlld(WL, WR, 0, g)
    flip = np.array([1, -1, 1, 1, 1, -1, 1, 1.0])
    F2, S2 = O.hlld(WR * flip, WL * flip, 0, g)
    sign = np.array([-1, 1, -1, -1, -1, -1, -1.0])
    assert np.allclose(F1, sign * F2, rtol=1e-12, atol=1e-14)


def _wave_error(kind, N, riemann):
    lay = ics.cartesian((2, 2, 1), (N // 2, N // 2, 4), dx=1.0 / N)
    W0 = np.array([1.0, 0, 0, 0, 0.6, 1.0, 0, 0])
    amp = 1e-6
    f = ics.linear_modes(lay, [(kind, (1, 1, 0), 0.3)], W0, G53, amp)
    _, lam = ics.eigenmode(W0, np.array([1, 1, 0]) / np.sqrt(2), G53, kind)
    T = (1 / np.sqrt(2)) / lam
    o = run(lay, f, t_end=T, time_mode=0, riemann=riemann)
    ref = ics.to_patches(lay, f)
    e = [np.mean(np.abs(a - b)) for a, b in zip(o.get_state(), ref)]
    return np.mean(e) / amp


@pytest.mark.parametrize("kind", ["fast", "alfven", "slow"])
def test_hlld_update_converges_at_second_order(kind):
    e32, e64 = _wave_error(kind, 32, 1), _wave_error(kind, 64, 1)
    assert np.log2(e32 / e64) >= 1.8, (e32, e64)


def test_hlld_keeps_a_stationary_contact_and_solves_sod():
    """A density step at rest in uniform pressure and field is a steady
    contact: with HLLD every face flux is the exact one, so the full update
    keeps it to rounding, where HLL smears it.  The Sod tube (B = 0, where
    HLLD is HLLC) converges to the exact solution no worse than with HLL."""
    lay = ics.cartesian((4, 1, 1), (16, 8, 8))
    rho = lambda x, y, z: np.where((x > 0.25) & (x < 0.75), 0.3, 1.0) + 0 * y
    state = ics.patches_from_functions(
        lay, rho, lambda x, y, z: (0 * x, 0 * x, 0 * x), lambda x, y, z: 0.6 + 0 * x, G53,
        faces=(lambda x, y, z: 0.5 + 0 * x, lambda x, y, z: 0.3 + 0 * x, lambda x, y, z: 0 * x))
    change = {}
    for r in (0, 1):
        o = run_state(lay, state, riemann=r, steps=20)
        change[r] = np.max(np.abs(o.get_state()[0] - state[0]))
    assert change[1] <= 1e-12 and change[0] > 1e-3, change
    errs = {}
    for r in (0, 1):
        lay, f = ics.config_sod(0, 256, cells_per_patch=64)
        o = run(lay, f, t_end=0.2, time_mode=0, riemann=r)
        Ug, *_ = ics.from_patches(lay, *o.get_state())
        rho = np.moveaxis(Ug[0], 2, -1)[0, 0]
        dx = 1.0 / 256
        x = (np.arange(rho.size) + 0.5) * dx
        win = (x >= 1.0) & (x < 2.0)
        ex = RX.sample((x[win] - 1.5) / 0.2, 1, 0, 1, 0.125, 0, 0.1, 1.4)[0]
        errs[r] = np.sum(np.abs(rho[win] - ex)) * dx
    assert errs[1] <= errs[0], errs


def run_state(lay, state, riemann, steps):
    from oracle import Oracle
    o = Oracle(lay.n, lay.lo, gamma=G53, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
               riemann=riemann)
    o.set_state(*state)
    o.advance(max_sweeps=steps)
    return o


def _normal(v7_lab, d):
    """Lab-order flux (mass, m_x, m_y, m_z, E, B_t1, B_t2) to the normal
    frame (mass, m_n, m_t1, m_t2, E, B_t1, B_t2)."""
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    return np.array([v7_lab[0], v7_lab[1 + d], v7_lab[1 + t1], v7_lab[1 + t2], v7_lab[4], v7_lab[5], v7_lab[6]])


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlld_fan_is_consistent_with_the_integral_form(d):
    """For general states: the fan's wave speeds times its jumps add up to
    F_R - F_L (the integral form over the fan), density and normal velocity
    do not jump across the rotational waves, and across the contact only
    density and energy jump (normal velocity, tangential velocity and field
    continuous); the outer waves give both star states the normal momentum
    flux of one total pressure pT*."""
    rng = np.random.default_rng(10 + d)
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    checked = 0
    for _ in range(40):
        W = [np.array([0.4 + rng.random(), *(0.7 * rng.standard_normal(3)), 0.2 + rng.random(),
                       *(rng.standard_normal(3))]) for _ in range(2)]
        W[1][5 + d] = W[0][5 + d]
        fan = O.hlld_fan(W[0], W[1], d, G53)
        if fan is None:
            continue
        S, U, pts = fan
        cU = lambda Wx: (lambda V: _normal(np.concatenate([V[:5], [V[5 + t1], V[5 + t2]]]), d))(cons(Wx, G53))
        UL, UR = cU(W[0]), cU(W[1])
        FL, FR = _normal(phys_flux(W[0], d, G53), d), _normal(phys_flux(W[1], d, G53), d)
        states = [UL, U[0], U[1], U[2], U[3], UR]
        total = sum(S[k] * (states[k + 1] - states[k]) for k in range(5))
        scale = np.max(np.abs(FR)) + np.max(np.abs(FL)) + 1.0
        assert np.max(np.abs(total - (FR - FL))) <= 1e-12 * scale
        assert U[0][0] == U[1][0] and U[3][0] == U[2][0]                  # rho across S*
        for k in range(4):
            assert U[k][1] / U[k][0] == pytest.approx(S[2], rel=1e-13, abs=1e-13)   # u = S_M
        v2 = [U[k][2:4] / U[k][0] for k in (1, 2)]
        assert np.allclose(v2[0], v2[1], rtol=1e-13, atol=1e-13)       # tangential v across S_M
        assert np.allclose(U[1][5:], U[2][5:], rtol=1e-13, atol=1e-13)  # tangential B across S_M
        # the outer waves' jump conditions give each star state the normal
        # momentum flux rho* S_M^2 + pT* - Bn^2 with one pT* on both sides
        bn = W[0][5 + d]
        for k, (Sa, Ua, Fa) in enumerate(((S[0], UL, FL), (S[4], UR, FR))):
            Us = U[0] if k == 0 else U[3]
            Fm = Fa[1] + Sa * (Us[1] - Ua[1])
            assert Fm == pytest.approx(Us[0] * S[2] ** 2 + pts - bn * bn, rel=1e-12, abs=1e-12 * scale)
        checked += 1
    assert checked >= 20


def hllc_toro(WL, WR, d, g, SL, SR):
    """The textbook HLLC flux (Toro, Riemann Solvers and Numerical Methods
    for Fluid Dynamics, the HLLC chapter: star states from the contact speed
    S* of the two outer jump conditions) for hydrodynamic states (rho, v, p)
    along axis d, given the outer speeds."""
    t1, t2 = (d + 1) % 3, (d + 2) % 3

    def parts(W):
        r, p = W[0], W[4]
        u, v, w = W[1 + d], W[1 + t1], W[1 + t2]
        E = p / (g - 1) + 0.5 * r * (u * u + v * v + w * w)
        U = np.array([r, r * u, r * v, r * w, E])
        F = np.array([r * u, r * u * u + p, r * u * v, r * u * w, (E + p) * u])
        return r, u, v, w, p, E, U, F

    rL, uL, vL, wL, pL, EL, UL, FL = parts(WL)
    rR, uR, vR, wR, pR, ER, UR, FR = parts(WR)
    Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def star(r, u, v, w, p, E, S):
        k = r * (S - u) / (S - Ss)
        return k * np.array([1.0, Ss, v, w, E / r + (Ss - u) * (Ss + p / (r * (S - u)))])

    if SL >= 0:
        F = FL
    elif Ss >= 0:
        F = FL + SL * (star(rL, uL, vL, wL, pL, EL, SL) - UL)
    elif SR > 0:
        F = FR + SR * (star(rR, uR, vR, wR, pR, ER, SR) - UR)
    else:
        F = FR
    out = np.empty(5)
    out[0], out[1 + d], out[1 + t1], out[1 + t2], out[4] = F
    return out


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlld_without_field_is_hllc(d):
    """With B = 0 the Alfven waves fall onto the contact and HLLD reduces to
    HLLC: random subsonic and supersonic hydrodynamic pairs along each axis
    give Toro's HLLC flux (same outer speeds) to 1e-13 of the flux scale."""
    rng = np.random.default_rng(40 + d)
    for _ in range(200):
        WL = np.zeros(8)
        WR = np.zeros(8)
        for W in (WL, WR):
            W[0] = rng.uniform(0.1, 3.0)
            W[1:4] = rng.normal(0.0, 1.5, 3)
            W[4] = rng.uniform(0.05, 3.0)
        F, S = O.hlld(WL, WR, d, G53)
        ref = hllc_toro(WL, WR, d, G53, S[0], S[1])
        scale = max(np.max(np.abs(ref)), 1.0)
        assert np.max(np.abs(F[:5] - ref)) <= 1e-13 * scale, (F[:5], ref)
        assert np.all(F[5:] == 0.0)
