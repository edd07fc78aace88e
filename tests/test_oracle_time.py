"""Pins of the oracle's readiness with grace and its time inter- and
extrapolation of guard values (DISPATCH I, Sec. 3 B: Eq. 1 with g > 0,
linear or higher-order time inter- and extrapolation from the stored
slices):

* guard values from a neighbour whose slices vary linearly (quadratically)
  in time are exact under linear (quadratic) inter- and extrapolation,
  between any two stored slices, past the newest one and at a slice time;
  quadratic data under linear interpolation are not;
* Eq. 1 with g > 0 lets a patch step while up to g times a neighbour's
  last step ahead of it, and not further; guard values are then
  extrapolated;
* a patch does not overwrite its oldest slice while a neighbour that may
  step first still needs it, and steps once a free slot exists;
* with power-of-two steps aligned to their size, g < 1 changes the local
  step input's schedule and state little or not at all;
* invalid combinations are rejected."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1705_10774_gb300 import ics

G53 = 5.0 / 3.0


def row_layout(npatch=2, n=8):
    return ics.cartesian((npatch, 1, 1), n)


def slice_data(lay, ip, phase, seed=0):
    """A physically valid slice of patch ip that is affine in `phase`:
    base + phase * pattern for every stored value."""
    rng = np.random.default_rng(100 + 7 * ip + seed)
    nx, ny, nz = (int(v) for v in lay.n[ip])
    nc = nx * ny * nz
    U = np.empty((5, nc))
    U[0] = 1.0 + 0.2 * rng.random(nc) + 0.1 * phase * rng.random(nc)
    U[1:4] = 0.1 * rng.standard_normal((3, nc)) * (1.0 + phase)
    U[4] = 3.0 + 0.1 * rng.random(nc) + 0.2 * phase * rng.random(nc)
    fx = 0.3 + 0.05 * rng.standard_normal((nx + 1) * ny * nz) * (1.0 + phase)
    fy = 0.1 * rng.standard_normal(nx * (ny + 1) * nz) * (1.0 + 0.5 * phase)
    fz = 0.1 * rng.standard_normal(nx * ny * (nz + 1)) * (1.0 - 0.3 * phase)
    return U.ravel(), fx, fy, fz


def setup_two(order, times, tP, poly, nslices=4, grace=0.5):
    """Patch 0 at tP (one slice); patch 1 with slices at `times` whose data
    follow poly(t); returns the oracle and the padded box of patch 0."""
    lay = row_layout()
    o = Oracle(lay.n, lay.lo, gamma=G53, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1,
               nslices=nslices, grace=grace, time_order=order)
    o.set_slot(0, 0, tP, *slice_data(lay, 0, 0.0))
    o.set_latest(0, 0, 0.0)
    for s, t in enumerate(times):
        o.set_slot(1, s, t, *slice_data(lay, 1, poly(t)))
    o.set_latest(1, len(times) - 1, times[-1] - times[-2])
    return lay, o, o.fill_padded(0)


def reference(lay, tP, poly, order):
    """The same padded box with patch 1 holding one slice at tP whose data
    is poly(tP) exactly (every guard value a plain copy)."""
    o = Oracle(lay.n, lay.lo, gamma=G53, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1,
               nslices=4, time_order=order)
    o.set_slot(0, 0, tP, *slice_data(lay, 0, 0.0))
    o.set_latest(0, 0, 0.0)
    o.set_slot(1, 0, tP, *slice_data(lay, 1, poly(tP)))
    o.set_latest(1, 0, 0.0)
    return o.fill_padded(0)


TIMES = [0.0, 0.25, 0.5, 1.0]
QUERY = [0.375, 0.75, 0.5, 1.1, 1.25]   # between slices, a slice time, past the newest


@pytest.mark.parametrize("tP", QUERY)
def test_linear_time_interpolation_and_extrapolation_are_exact_for_linear_data(tP):
    poly = lambda t: 0.3 + 0.8 * t
    lay, _, got = setup_two(1, TIMES, tP, poly)
    want = reference(lay, tP, poly, 1)
    for a, b in zip(got, want):
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))


@pytest.mark.parametrize("tP", QUERY)
def test_quadratic_time_interpolation_and_extrapolation_are_exact_for_quadratic_data(tP):
    poly = lambda t: 0.3 + 0.8 * t - 0.9 * t * t
    lay, _, got = setup_two(2, TIMES, tP, poly)
    want = reference(lay, tP, poly, 2)
    for a, b in zip(got, want):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    if tP not in TIMES:
        # the linear form misses the curvature
        _, _, lin = setup_two(1, TIMES, tP, poly)
        assert max(np.max(np.abs(a - b)) for a, b in zip(lin, want)) > 1e-4


def chain_state(lay, times, dts, nslices=3, grace=0.3, order=1, extra_slices=None):
    """Patches in a row with given current times and last steps; each holds
    its current slice and the slice one last step earlier (extra_slices
    adds more: {patch: [times]})."""
    o = Oracle(lay.n, lay.lo, gamma=G53, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1,
               nslices=nslices, grace=grace, time_order=order)
    for ip, (t, dt) in enumerate(zip(times, dts)):
        ts = sorted(set((extra_slices or {}).get(ip, []) + [t - dt, t]))
        for s, ti in enumerate(ts):
            o.set_slot(ip, s, ti, *slice_data(lay, ip, 0.1 * ti))
        o.set_latest(ip, len(ts) - 1, dt)
    return o


def test_grace_lets_a_patch_step_within_g_of_a_neighbours_step():
    """Four patches in a periodic row, P1 at 1.25 (last step 0.25) between
    P0 at 1.0 (last step 1.0) and P2 at 1.5: with g = 0 P1 waits for P0;
    with g = 0.3 it may run 0.3 ahead of P0 and steps, its guard values from
    P0 extrapolated; P0 itself waits for P3 at 0.5 either way."""
    lay = row_layout(4)
    times, dts = [1.0, 1.25, 1.5, 0.5], [1.0, 0.25, 1.0, 0.5]
    stepped = {}
    for g in (0.0, 0.3):
        o = chain_state(lay, times, dts, grace=g)
        o.advance(max_sweeps=1)
        t = o.get_times()[0]
        stepped[g] = t > np.array(times)
    assert not stepped[0.0][1] and stepped[0.3][1]
    assert not stepped[0.0][0] and not stepped[0.3][0]
    assert stepped[0.0][3] and stepped[0.3][3]


def test_grace_limit_is_g_times_the_neighbours_last_step():
    """P1 1.25 ahead-of-P0 distance 0.25 needs g >= 0.25 with P0's last
    step 1.0: g = 0.2 keeps it waiting, g = 0.25 lets it go."""
    lay = row_layout(4)
    times, dts = [1.0, 1.25, 1.5, 0.5], [1.0, 0.25, 1.0, 0.5]
    go = []
    for g in (0.2, 0.25):
        o = chain_state(lay, times, dts, grace=g)
        o.advance(max_sweeps=1)
        go.append(o.get_times()[0][1] > 1.25)
    assert go == [False, True]


def test_oldest_slice_is_kept_while_a_neighbour_needs_it():
    """P1 (slices 1.0, 1.125, 1.25; three slots) may run ahead of P0 at 1.0
    by Eq. 1, but P0 still needs P1's slice at 1.0, the one P1 would
    overwrite: P1 waits.  With a fourth slot free it steps."""
    lay = row_layout(4)
    times, dts = [1.0, 1.25, 1.5, 0.5], [1.0, 0.125, 1.0, 0.5]
    res = []
    for ns in (3, 4):
        o = chain_state(lay, times, dts, nslices=ns, grace=0.3, extra_slices={1: [1.0]})
        o.advance(max_sweeps=1)
        res.append(o.get_times()[0][1] > 1.25)
    assert res == [False, True]


def lts_run(grace, order=1, nslices=3):
    lay, f = ics.config_lts(patches=8, n=4, sigma_ln=2.0, hot_radius=0.2, hot_factor=300.0)
    o = Oracle(lay.n, lay.lo, gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1,
               grace=grace, time_order=order, nslices=nslices)
    o.set_state(*ics.to_patches(lay, f))
    o.advance(t_end=0.002)
    return o


def test_grace_on_aligned_power_of_two_steps_changes_little():
    """Steps that are powers of two aligned to their size leave g < 1 little
    room (a patch may run ahead only of a neighbour whose step is at least
    1/g times its own, and only while a third patch holds that neighbour):
    on the local-step input (512 patches, steps spanning a factor > 200)
    g = 0.3 gives the g = 0 schedule and state, and g = 0.6 and quadratic
    time interpolation stay within 1e-6 relative L1; all runs complete
    (the oldest patch can always step)."""
    ref = lts_run(0.0)
    a = ref.get_state()
    key = lambda s: sorted(zip(*(x.tolist() for x in s)))
    o3 = lts_run(0.3)
    assert key(o3.schedule()) == key(ref.schedule())
    assert all(np.array_equal(x, y) for x, y in zip(o3.get_state(), a))
    for o in (lts_run(0.6), lts_run(0.0, order=2), lts_run(0.3, order=2, nslices=4)):
        b = o.get_state()
        num = sum(float(np.abs(x - y).sum()) for x, y in zip(a, b))
        den = sum(float(np.abs(x).sum()) for x in a)
        assert num / den <= 1e-6
        assert np.all(o.get_times()[0] == 0.002)


def test_time_parameters_are_validated():
    lay = row_layout()
    base = dict(gamma=G53, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    for bad in (dict(grace=1.0), dict(grace=-0.1), dict(time_order=3), dict(grace=0.3, time_mode=1, dispatcher=0),
                dict(grace=0.3, time_order=2, nslices=3)):
        with pytest.raises(Exception):
            Oracle(lay.n, lay.lo, **base, **bad)
    Oracle(lay.n, lay.lo, **base, grace=0.3, time_order=2, nslices=4, time_mode=1)


# which slices: the error of data one degree too high names them
WINDOWS = {  # query time -> (linear pair, quadratic triple), older first
    0.375: ((0.25, 0.5), (0.0, 0.25, 0.5)),
    0.75: ((0.5, 1.0), (0.25, 0.5, 1.0)),
    1.1: ((0.5, 1.0), (0.25, 0.5, 1.0)),
    1.25: ((0.5, 1.0), (0.25, 0.5, 1.0)),
    0.125: ((0.0, 0.25), (0.0, 0.25, 0.5)),
}


@pytest.mark.parametrize("tP", sorted(WINDOWS))
def test_the_slices_used_are_the_documented_ones(tP):
    """Linear inter- and extrapolation of quadratic data c t^2 misses by
    -c (t - t_a)(t - t_b), quadratic of cubic data d t^3 by
    -d (t - t_a)(t - t_b)(t - t_c): the measured miss names the slices.
    Linear: the two slices around t, or the newest two past the newest.
    Quadratic: those two and the next older slice (the next newer where
    none is older), or the newest three past the newest."""
    lay = row_layout()
    pattern = [a - b for a, b in zip(reference(lay, tP, lambda t: 1.0, 1), reference(lay, tP, lambda t: 0.0, 1))]
    for order, poly, coef in ((1, lambda t: 0.7 * t * t, 0.7), (2, lambda t: -0.6 * t ** 3, -0.6)):
        _, _, got = setup_two(order, TIMES, tP, poly)
        want = reference(lay, tP, poly, order)
        num = sum(float(np.sum((a - b) * q)) for a, b, q in zip(got, want, pattern))
        den = sum(float(np.sum(q * q)) for q in pattern)
        win = WINDOWS[tP][order - 1]
        expect = -coef * np.prod([tP - s for s in win])
        assert abs(num / den - expect) <= 1e-10, (order, num / den, expect)
