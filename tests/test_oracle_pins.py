"""Pins of the FP64 oracle against what mathematics and physics fix.

None of these compares the oracle with itself: each check uses a closed form,
an independently built linearisation (the primitive Jacobian of ideal MHD,
diagonalised by a library routine), an exact Riemann solution, an invariant
of the discrete scheme (conservation, div B, uniform states) or a structural
identity of the dispatcher (local = global stepping when all steps agree;
sweep = time-sorted queue).  A dropped term, a wrong sign or a transposed
index in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from oracle import oracle as O
from paper_1705_10774_gb300 import ics
import riemann_exact as RX

G53 = 5.0 / 3.0
HERE = os.path.dirname(os.path.abspath(__file__))


def cons(W, gamma):
    """Conserved variables (rho, m, E, B) of a primitive state (definition)."""
    rho, v, p, B = W[0], W[1:4], W[4], W[5:8]
    E = p / (gamma - 1) + 0.5 * rho * np.dot(v, v) + 0.5 * np.dot(B, B)
    return np.concatenate([[rho], rho * v, [E], B])


def run(lay, f, steps=None, t_end=np.inf, **kw):
    o = Oracle(lay.n, lay.lo, gamma=f.gamma, cfl=kw.pop("cfl", 0.4), base_cells=lay.base_cells,
               box_len=lay.box_len, **kw)
    o.set_state(*ics.to_patches(lay, f))
    if steps != 0:
        o.advance(t_end=t_end, max_sweeps=steps or 0)
    return o


# ------------------------------------------------------------ cell level

def test_mc_limiter_cases():
    assert O.mc(1.0, 2.0) == 1.5            # central slope wins
    assert O.mc(1.0, 10.0) == 2.0           # twice the smaller one-sided slope
    assert O.mc(-1.0, -3.0) == -2.0
    assert O.mc(1.0, -1.0) == 0.0           # extremum
    assert O.mc(0.0, 1.0) == 0.0
    assert O.mc(3.0, 1.0) == 2.0
    rng = np.random.default_rng(0)
    for dl, dr in rng.standard_normal((200, 2)):
        s = O.mc(dl, dr)
        if dl * dr > 0:   # TVD bounds: same sign, |s| <= 2 min(|dl|,|dr|), |s| <= |dl+dr|/2
            assert np.sign(s) == np.sign(dl)
            assert abs(s) <= 2 * min(abs(dl), abs(dr)) and abs(s) <= 0.5 * abs(dl + dr) + 1e-15
        else:
            assert s == 0.0


def test_pow2_floor_exact():
    for x, want in [(0.3, 0.25), (1.0, 1.0), (0.75, 0.5), (2.0 ** -20, 2.0 ** -20),
                    (np.nextafter(1.0, 0.0), 0.5), (3.0e-7, 2.0 ** -22), (1000.0, 512.0)]:
        assert O.pow2_floor(x) == want


def test_fast_speed_closed_forms():
    g = G53
    rho, p = 1.3, 0.7
    a = np.sqrt(g * p / rho)
    assert O.cfast(g, rho, p, 0, 0, 0) == pytest.approx(a, rel=1e-15)
    # field along the normal: c_f = max(a, v_A)
    for b in (0.3, 2.0):
        assert O.cfast(g, rho, p, b, 0, 0) == pytest.approx(max(a, b / np.sqrt(rho)), rel=1e-14)
    # field normal to the direction: c_f^2 = a^2 + v_A^2
    assert O.cfast(g, rho, p, 0, 0.4, 0.9) == pytest.approx(np.sqrt(a * a + (0.16 + 0.81) / rho), rel=1e-14)


@pytest.mark.parametrize("khat", [(1, 0, 0), (0.6, 0.8, 0), (1 / np.sqrt(3),) * 3])
def test_jacobian_speeds_match_closed_forms(khat):
    """The independently written primitive Jacobian has the textbook speeds;
    the oracle's fast speed equals its largest eigenvalue."""
    W0 = np.array([1.2, 0, 0, 0, 0.8, 0.9, 0.5, -0.3])
    g = G53
    kh = np.asarray(khat, float)
    lam = np.sort(np.linalg.eigvals(ics.primitive_jacobian(W0, kh, g)).real)
    rho, p, B = W0[0], W0[4], W0[5:8]
    a2 = g * p / rho
    b2 = B @ B / rho
    bn2 = (B @ kh) ** 2 / rho
    cf = np.sqrt(0.5 * (a2 + b2 + np.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)))
    cs = np.sqrt(0.5 * (a2 + b2 - np.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)))
    ca = np.sqrt(bn2)
    assert np.allclose(lam, np.sort([-cf, -ca, -cs, 0, 0, cs, ca, cf]), atol=1e-12)
    bn = B @ kh
    bt = B - bn * kh
    assert O.cfast(g, rho, p, bn, np.linalg.norm(bt), 0.0) == pytest.approx(cf, rel=1e-13)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("kind", ["fast", "alfven", "slow"])
def test_hll_flux_matches_linearised_jump(d, kind):
    """F(W) = hll(W, W) is the physical flux: across a small-amplitude
    eigenmode of A(e_d) its jump equals the wave speed times the jump of the
    conserved variables (all seven components, magnetic terms included)."""
    g = G53
    W0 = np.array([1.1, 0.3, -0.2, 0.15, 0.9, 0.7, 0.4, -0.5])
    kh = np.eye(3)[d]
    r, lam = ics.eigenmode(W0, kh, g, kind)
    eps = 1e-5
    Wp, Wm = W0 + eps * r, W0 - eps * r
    Fp, Sp = O.hll(Wp, Wp, d, g)
    Fm, _ = O.hll(Wm, Wm, d, g)
    Up, Um = cons(Wp, g), cons(Wm, g)
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    dU = np.concatenate([(Up - Um)[:5], [(Up - Um)[5 + t1], (Up - Um)[5 + t2]]])
    dF = Fp - Fm
    assert np.allclose(dF, lam * dU, atol=1e-9 * eps, rtol=1e-6)
    assert Sp[0] < 0 < Sp[1] or np.all(np.abs(W0[1:4]) > 10)


def test_hll_upwind_and_mirror_symmetry():
    g = 1.4
    WL = np.array([1.0, 5.0, 0.1, 0.0, 1.0, 0.2, 0.1, 0.0])
    WR = np.array([0.8, 5.2, 0.0, 0.1, 0.9, 0.2, 0.0, 0.1])
    F, S = O.hll(WL, WR, 0, g)
    Fl, _ = O.hll(WL, WL, 0, g)
    assert S[0] > 0 and np.array_equal(F, Fl)      # supersonic: upwind state only
    # mirror x -> -x: swap sides, flip normal velocity and normal field
    WL2 = np.array([1.0, 0.2, 0.1, 0.0, 1.0, 0.5, 0.1, 0.3])
    WR2 = np.array([0.5, -0.3, 0.0, 0.1, 0.4, 0.5, -0.2, 0.1])
    F1, S1 = O.hll(WL2, WR2, 0, g)
    flip = np.array([1, -1, 1, 1, 1, -1, 1, 1.0])
    F2, S2 = O.hll(WR2 * flip, WL2 * flip, 0, g)
    sign = np.array([-1, 1, -1, -1, -1, -1, -1.0])   # only the normal-momentum flux keeps its sign
    assert np.allclose(F1, sign * F2, rtol=1e-13, atol=1e-15)
    assert S1[0] == pytest.approx(-S2[1]) and S1[1] == pytest.approx(-S2[0])


def test_emf_reduces_to_hll_induction_flux_in_1d():
    """With no variation along y the upwind edge EMF is minus the HLL flux of
    B_y through the x-face."""
    g = G53
    rng = np.random.default_rng(3)
    for _ in range(20):
        WL = np.array([1.0, 0.3, -0.1, 0.2, 0.8, 0.6, 0.2, -0.1]) + 0.1 * rng.standard_normal(8)
        WR = np.array([0.7, -0.2, 0.3, 0.0, 0.5, 0.6, -0.4, 0.3]) + 0.1 * rng.standard_normal(8)
        WR[5] = WL[5]
        F, S = O.hll(WL, WR, 0, g)
        apx, amx = max(0.0, S[1]), max(0.0, -S[0])
        apy, amy = 0.7, 0.4
        Ez = O.emf(WL, WR, WL, WR, 2, apx, amx, apy, amy)
        assert Ez == pytest.approx(-F[5], rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("kind", ["fast", "alfven", "slow"])
def test_predictor_advances_a_linear_wave(kind):
    """With slopes of a plane eigenmode, dW_d = eps khat_d r, the half-step
    predictor moves W by -h eps lambda r (to second order in eps)."""
    g = G53
    W0 = np.array([1.0, 0.2, -0.1, 0.05, 0.6, 1.0, 0.3, -0.2])
    kh = np.array([0.48, 0.6, 0.64])
    r, lam = ics.eigenmode(W0, kh, g, kind)
    eps, h = 1e-6, 0.37
    Ws = O.predict(W0, eps * kh[0] * r, eps * kh[1] * r, eps * kh[2] * r, g, h)
    assert np.allclose((Ws - W0) / (h * eps), -lam * r, atol=1e-6)


def test_primitive_roundtrip():
    g = G53
    W = np.array([1.3, 0.4, -0.2, 0.1, 0.9, 0.5, -0.6, 0.2])
    U = cons(W, g)
    faces = [0.45, 0.55, -0.7, -0.5, 0.1, 0.3]     # means are (0.5, -0.6, 0.2)
    Wp = O.prim(U[:5], faces, g)
    assert np.allclose(Wp, W, rtol=1e-14, atol=1e-15)


def test_exact_riemann_solver_against_published_star_state():
    vals = {}
    with open(os.path.join(HERE, "golden", "sod_star_state.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    ps, us = RX.star_state(1, 0, 1, 0.125, 0, 0.1, 1.4)
    assert ps == pytest.approx(vals["p_star"], abs=6e-6)
    assert us == pytest.approx(vals["u_star"], abs=6e-6)
    rl, _, _ = RX.sample(np.array([0.5]), 1, 0, 1, 0.125, 0, 0.1, 1.4)
    rr, _, _ = RX.sample(np.array([1.5]), 1, 0, 1, 0.125, 0, 0.1, 1.4)
    assert rl[0] == pytest.approx(vals["rho_star_left"], abs=6e-6)
    assert rr[0] == pytest.approx(vals["rho_star_right"], abs=6e-6)


# ------------------------------------------------------------ scheme level

def test_uniform_state_is_exactly_steady():
    lay = ics.cartesian(2, 6)
    f = ics.config_uniform(lay, [1.3, 0.4, -0.7, 0.2, 0.8, 0.6, -0.3, 0.9], G53)
    o = run(lay, f, steps=5)
    U, bx, by, bz = o.get_state()
    U0, bx0, by0, bz0 = ics.to_patches(lay, f)
    assert np.array_equal(U, U0) and np.array_equal(bx, bx0)
    assert np.array_equal(by, by0) and np.array_equal(bz, bz0)


def _turbulent_small(seed=5, patches=2, n=8, mach=1.0):
    lay, f = ics.config_turbulence(seed=seed, patches=patches, n=n, mach=mach)
    rng = np.random.default_rng(seed + 1)
    X, Y, Z = lay.base_cells
    A = [ics.gaussian_filtered_noise((Z, Y, X), lay.box_len, 0.1, rng) * 0.02 for _ in range(3)]
    dbx, dby, dbz = ics.curl_faces(A[0], A[1], A[2], lay.dx)
    f.bx = f.bx + dbx; f.by = f.by + dby; f.bz = f.bz + dbz
    return lay, f


def test_conservation_and_divb_on_periodic_box():
    lay, f = _turbulent_small()
    o0 = run(lay, f, steps=0)
    d0 = o0.diagnostics()
    steps = 12
    o = run(lay, f, steps=steps)
    d1 = o.diagnostics()
    U, bx, by, bz = o.get_state()
    dV = lay.dx ** 3
    Uabs = np.abs(U.reshape(-1)).sum() * dV
    tol = 1e-13 * steps * Uabs
    assert abs(d1["mass"] - d0["mass"]) <= tol
    assert abs(d1["energy"] - d0["energy"]) <= tol
    assert np.all(np.abs(d1["mom"] - d0["mom"]) <= tol)
    assert np.all(np.abs(d1["bmean"] - d0["bmean"]) <= tol)
    assert d1["max_divb"] <= 1e-13 * d1["max_b"]
    assert o.stats()["fallbacks"] == 0
    # the state did change
    assert not np.allclose(U, ics.to_patches(lay, f)[0])


def test_divb_survives_local_time_steps():
    """Each patch owns every face of its cells, so div b stays at round-off
    even when neighbours run different steps."""
    lay, f = ics.config_lts(patches=6, n=4, sigma_ln=1.0, hot_radius=0.15, hot_factor=100.0)
    o = run(lay, f, t_end=0.003, time_mode=1, dispatcher=1)
    d = o.diagnostics()
    assert d["max_divb"] <= 1e-13 * d["max_b"]
    dts = o.schedule()[2]
    pow2 = dts[np.exp2(np.floor(np.log2(dts))) == dts]
    assert len(np.unique(pow2)) >= 3


def test_local_equals_global_when_steps_agree():
    lay = ics.cartesian(2, 8)
    f = ics.config_uniform(lay, [1.0, 0.1, 0.0, -0.05, 0.6, 0.7, 0.2, 0.0], G53, seed=11, eps=1e-8)
    og = run(lay, f, steps=6, time_mode=0)
    t_end = og.get_times()[0][0]
    ol = run(lay, f, t_end=t_end, time_mode=1, dispatcher=1)
    oq = run(lay, f, t_end=t_end, time_mode=1, dispatcher=0)
    sg, sl, sq = og.schedule(), ol.schedule(), oq.schedule()
    key = lambda s: sorted(zip(s[0].tolist(), s[1].tolist(), s[2].tolist()))
    assert key(sg) == key(sl) == key(sq)
    for a, b in zip(og.get_state(), ol.get_state()):
        assert np.array_equal(a, b)
    for a, b in zip(og.get_state(), oq.get_state()):
        assert np.array_equal(a, b)


def test_sweep_equals_time_sorted_queue_under_local_steps():
    lay, f = ics.config_lts(patches=6, n=4, sigma_ln=1.0, hot_radius=0.15, hot_factor=100.0)
    t_end = 0.003
    os_ = run(lay, f, t_end=t_end, time_mode=1, dispatcher=1)
    oq = run(lay, f, t_end=t_end, time_mode=1, dispatcher=0)
    ss, sq = os_.schedule(), oq.schedule()
    key = lambda s: sorted(zip(s[0].tolist(), s[1].tolist(), s[2].tolist()))
    assert key(ss) == key(sq)
    for a, b in zip(os_.get_state(), oq.get_state()):
        assert np.array_equal(a, b)
    # the run really used several step sizes, and the schedule is consistent
    p, t, dt = ss
    assert len(np.unique(dt)) >= 3
    for ip in range(lay.npatch):
        sel = p == ip
        tt, dd = t[sel], dt[sel]
        assert np.all(tt[1:] == tt[:-1] + dd[:-1])          # contiguous in time
        assert tt[-1] + dd[-1] == t_end
        full = dd[:-1]
        assert np.all(np.exp2(np.floor(np.log2(full))) == full)  # powers of two
        assert np.all(np.fmod(tt[:-1], full) == 0.0)             # aligned
    assert np.all(os_.get_times()[0] == t_end)


def _sod_profile(axis, npu, t_end=0.2, cpp=64):
    lay, f = ics.config_sod(axis, npu, cells_per_patch=cpp)
    o = run(lay, f, t_end=t_end, time_mode=0)
    Ug, *_ = ics.from_patches(lay, *o.get_state())
    rho = np.moveaxis(Ug[0], 2 - axis, -1)
    return rho[0, 0], lay


def test_sod_orientations_agree():
    r = [_sod_profile(ax, 64, t_end=0.1, cpp=32)[0] for ax in range(3)]
    assert np.allclose(r[0], r[1], rtol=1e-12, atol=1e-14)
    assert np.allclose(r[0], r[2], rtol=1e-12, atol=1e-14)


def test_sod_shock_tube_against_exact_solution():
    errs = []
    for npu in (128, 256, 512):
        rho, lay = _sod_profile(0, npu)
        dx = 1.0 / npu
        x = (np.arange(rho.size) + 0.5) * dx
        win = (x >= 1.0) & (x < 2.0)
        ex = RX.sample((x[win] - 1.5) / 0.2, 1, 0, 1, 0.125, 0, 0.1, 1.4)[0]
        errs.append(np.sum(np.abs(rho[win] - ex)) * dx)
        if npu == 256:
            # shock position: where the density crosses the post/pre-shock mean
            ps, us = RX.star_state(1, 0, 1, 0.125, 0, 0.1, 1.4)
            r2 = RX.sample(np.array([us + 1e-6]), 1, 0, 1, 0.125, 0, 0.1, 1.4)[0][0]
            mid = 0.5 * (r2 + 0.125)
            xs = x[win]
            right = xs > 1.5 + us * 0.2 + 0.02
            i = np.nonzero(right & (rho[win] < mid))[0][0]
            x_num = xs[i]
            g = 1.4
            Ms = np.sqrt((g + 1) / (2 * g) * ps / 0.1 + (g - 1) / (2 * g))
            x_ex = 1.5 + Ms * np.sqrt(g * 0.1 / 0.125) * 0.2
            assert abs(x_num - x_ex) <= 2 * dx
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order >= 0.6), (errs, order)


def _wave_error(kind, N):
    lay = ics.cartesian((2, 2, 1), (N // 2, N // 2, 4), dx=1.0 / N)
    W0 = np.array([1.0, 0, 0, 0, 0.6, 1.0, 0, 0])
    amp = 1e-6
    f = ics.linear_modes(lay, [(kind, (1, 1, 0), 0.3)], W0, G53, amp)
    _, lam = ics.eigenmode(W0, np.array([1, 1, 0]) / np.sqrt(2), G53, kind)
    T = (1 / np.sqrt(2)) / lam
    o = run(lay, f, t_end=T, time_mode=0)
    assert np.all(o.get_times()[0] == T)
    ref = ics.to_patches(lay, f)
    out = o.get_state()
    e = [np.mean(np.abs(a - b)) for a, b in zip(out, ref)]
    return np.mean(e) / amp


@pytest.mark.parametrize("kind", ["fast", "alfven", "slow"])
def test_linear_wave_second_order_convergence(kind):
    e = [_wave_error(kind, N) for N in (16, 32, 64)]
    order = np.log2(e[1] / e[2])
    assert order >= 1.8, (kind, e)


def test_guard_time_interpolation_weight_and_direction():
    """A neighbour holding slices at t_a = 0 and t_b = 4h, read by a patch at
    t = h: the guard value must be S_a + (1/4)(S_b - S_a).  With S_a = 1 and
    S_b = 2 the patch's own uniform interior (density 1.25) then sees a
    uniform state and its update leaves it exactly unchanged; a reversed or
    wrongly scaled weight makes the guards differ and the state move."""
    lay = ics.cartesian((2, 1, 1), (6, 6, 6))
    g = 5.0 / 3.0
    W = lambda rho: [rho, 0.0, 0.0, 0.0, 0.6, 0.0, 0.0, 0.0]
    def patch_state(rho):
        f = ics.config_uniform(ics.cartesian(1, 6), W(rho), g)
        return ics.to_patches(ics.cartesian(1, 6), f)
    h = 2.0 ** -10
    o = Oracle(lay.n, lay.lo, gamma=g, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1)
    o.set_state(*[np.concatenate([a, a]) for a in patch_state(1.25)])
    o.set_slot(0, 0, h, *patch_state(1.25))     # the patch at t = h
    o.set_latest(0, 0)
    o.set_slot(1, 0, 0.0, *patch_state(1.0))    # neighbour: t_a = 0 ...
    o.set_slot(1, 1, 4 * h, *patch_state(2.0))  # ... and t_b = 4h (newest)
    o.set_latest(1, 1)
    U, bx, by, bz, _ = o.update_patch(0, h)
    U0 = patch_state(1.25)[0]
    assert np.array_equal(U, U0)
    # the same patch next to a neighbour whose interpolated value differs moves
    o.set_slot(1, 1, 4 * h, *patch_state(3.0))
    U2 = o.update_patch(0, h)[0]
    assert not np.array_equal(U2, U0)


def test_mc_limiter_sign_test_does_not_underflow():
    """Differences of one sign whose product would underflow to zero still
    get a limited slope (the extremum test is a sign test), and the result
    scales with them."""
    for scale in (1e-170, 1e-200, 1e-300):
        s = O.mc(1.0 * scale, 2.0 * scale)
        assert s == 1.5 * scale
        assert O.mc(-1.0 * scale, -3.0 * scale) == -2.0 * scale
    assert O.mc(1e-200, -1e-200) == 0.0
    assert O.mc(-0.0, 1.0) == 0.0 and O.mc(1.0, -0.0) == 0.0


def test_pressure_floor_count():
    """The oracle counts the cells of new slices whose pressure recovery took
    the floor p >= 1e-20 rho.  A cold uniform state with dyadic values (p = 0
    exactly, E = rho v^2 / 2, B = 0) stays exactly uniform, so every new cell
    recovers p = 0 and takes the floor; a warm wave input never does."""
    lay = ics.cartesian(2, 8)
    f = ics.config_uniform(lay, [1.0, 0.5, -0.25, 0.125, 0.0, 0.0, 0.0, 0.0], 5.0 / 3.0)
    o = Oracle(lay.n, lay.lo, gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    o.set_state(*ics.to_patches(lay, f))
    o.advance(max_sweeps=3)
    st = o.stats()
    assert st["cell_updates"] == 3 * 8 * 8 ** 3
    assert st["floors"] == st["cell_updates"]
    lay, f = ics.config_linear_waves(n=8)
    o = Oracle(lay.n, lay.lo, gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    o.set_state(*ics.to_patches(lay, f))
    o.advance(max_sweeps=3)
    assert o.stats()["floors"] == 0
