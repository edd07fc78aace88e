"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

FP64: relative L-infinity per field <= 1e-11 (max|a-b| / max|b|); the FP64
kernels and the oracle evaluate the same operation sequence without FMA
contraction, so the expected difference is 0.  Schedules must be identical.
"""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch, DispatchError, DSP_ERR_UNSUPPORTED, DSP_ERR_INVALID_ARG, \
    DSP_ERR_UNPHYSICAL
from oracle import Oracle

from fields import NAMES, field_errors, split_fields

TOL64 = 1e-11


def rel_linf(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def kw_of(lay, f, **extra):
    d = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    d.update(extra)
    return d


def pair(lay, f, gpu_extra=None, **common):
    state = ics.to_patches(lay, f)
    ge = dict(sched_capacity=1 << 20)
    ge.update(gpu_extra or {})
    g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, **common), **ge)
    g.set_state(*state)
    o = Oracle(lay.n, lay.lo, **kw_of(lay, f, **common))
    o.set_state(*state)
    return g, o


def state_error(out, ref):
    """Relative L-infinity over the whole conserved state: the largest
    difference in any field over the largest magnitude of any field.  Used for
    the FMA build on inputs whose momentum and transverse field are pure
    1e-6 perturbations, where a per-field norm measures FP64 rounding of O(1)
    flux terms against the perturbation."""
    num = max(float(np.max(np.abs(a - b))) for a, b in zip(out, ref))
    den = max(float(np.max(np.abs(b))) for b in ref)
    return num / den


def assert_same(g, o, tol=TOL64, whole_state=False):
    """Relative L-infinity per field (rho, m_x, m_y, m_z, E, b_x, b_y, b_z),
    or over the whole state (see state_error), and equal patch times."""
    out = g.get_state()
    ref = o.get_state()
    if whole_state:
        assert state_error(out, ref) <= tol, state_error(out, ref)
    else:
        errs = field_errors(out, ref, np.prod(g.n, axis=1))
        assert max(errs.values()) <= tol, errs
    assert np.array_equal(g.times()[0], o.get_times()[0])


def test_linear_waves_global_step_bit_parity():
    """Eight 16^3 patches, four seeded linear modes, 20 global steps."""
    lay, f = ics.config_linear_waves()
    g, o = pair(lay, f, time_mode=0)
    st = g.advance(max_sweeps=20)
    o.advance(max_sweeps=20)
    assert st["patch_updates"] == 160 and st["cell_updates"] == 160 * 16 ** 3
    assert_same(g, o)
    gp, gt, gd = g.schedule()
    op, ot, od = o.schedule()
    assert np.array_equal(gp, op) and np.array_equal(gt, ot) and np.array_equal(gd, od)
    out = g.get_state()
    ref = o.get_state()
    assert all(np.array_equal(a, b) for a, b in zip(out, ref)), "expected bit-identical FP64 results"


@pytest.mark.parametrize("tile_z", [0, 3])
def test_ragged_tiles_and_non_cubic_patches(tile_z):
    """Patches of 20 x 12 x 10 cells: x spans a full and a partial tile, y a
    full and a partial one, and with tile_z = 3 the z runs end ragged too."""
    lay = ics.cartesian((2, 2, 2), (20, 12, 10), dx=1.0 / 40)
    rng = np.random.default_rng(9)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    v = ics.solenoidal_velocity(shape, lay.box_len, 1.0, 3.0, 1.2, rng)
    A = [ics.gaussian_filtered_noise(shape, lay.box_len, 0.08, rng) * 0.01 for _ in range(3)]
    bx, by, bz = ics.curl_faces(*A, lay.dx)
    f = ics.Fields(rho=1.0 + 0.3 * ics.gaussian_filtered_noise(shape, lay.box_len, 0.1, rng) ** 2, v=v,
                   p=np.full(shape, 0.6), bx=bx + 0.5, by=by + 0.2, bz=bz, gamma=5.0 / 3.0)
    g, o = pair(lay, f, gpu_extra=dict(tile_z=tile_z), time_mode=0)
    g.advance(max_sweeps=6)
    o.advance(max_sweeps=6)
    assert_same(g, o)


def test_single_patch_is_its_own_neighbour():
    lay = ics.cartesian(1, 8)
    f = ics.config_uniform(lay, [1.0, 0.2, -0.1, 0.3, 0.6, 0.8, 0.1, -0.2], 5.0 / 3.0, seed=4, eps=1e-3)
    g, o = pair(lay, f, time_mode=0)
    g.advance(max_sweeps=5)
    o.advance(max_sweeps=5)
    assert_same(g, o)


@pytest.mark.parametrize("case", ["turbulence", "lts", "waves"])
def test_fp64_fma_form_within_tolerance(case):
    """FP64 with fused multiply-adds (precision 2): rounding differs from the
    oracle's; each conserved field must stay within 1e-11 relative L-infinity
    (rho, m_x, m_y, m_z, E, b_x, b_y, b_z on their own) on the turbulence
    input (20 global steps) and under local steps, and the schedule must be
    identical.  On the 1e-6-amplitude wave input the momentum and transverse
    field are pure perturbations, whose own maximum is 1e-6 of the O(1)
    flux terms whose rounding FMA changes, so there the norm is taken over
    the whole state."""
    if case == "lts":
        lay, f = _lts_case()
        common, run = dict(time_mode=1), dict(t_end=0.003)
    elif case == "turbulence":
        lay, f = ics.config_turbulence(seed=5, patches=2, n=16, mach=2.0)
        common, run = dict(time_mode=0), dict(max_sweeps=20)
    else:
        lay, f = ics.config_linear_waves()
        common, run = dict(time_mode=0), dict(max_sweeps=20)
    g, o = pair(lay, f, gpu_extra=dict(precision=2), **common)
    g.advance(**run)
    o.advance(**run)
    assert_same(g, o, whole_state=case == "waves")
    gp, gt, gd = g.schedule()
    op, ot, od = o.schedule()
    assert np.array_equal(gp, op) and np.array_equal(gt, ot) and np.array_equal(gd, od)


def _lts_case():
    return ics.config_lts(patches=6, n=4, sigma_ln=1.0, hot_radius=0.15, hot_factor=100.0)


def test_local_time_steps_schedule_and_state():
    """Local steps spanning a factor > 8: the GPU sweep dispatcher must
    reproduce the oracle's schedule entry by entry, and the states."""
    lay, f = _lts_case()
    g, o = pair(lay, f, time_mode=1, dispatcher=1)
    t_end = 0.003
    g.advance(t_end=t_end)
    o.advance(t_end=t_end)
    gp, gt, gd = g.schedule()
    op, ot, od = o.schedule()
    assert len(np.unique(od)) >= 3
    assert np.array_equal(gp, op) and np.array_equal(gt, ot) and np.array_equal(gd, od)
    assert_same(g, o)
    assert np.all(g.times()[0] == t_end)


def test_sweep_schedule_equals_time_sorted_queue():
    """The GPU sweep schedule equals the oracle's time-sorted queue schedule
    as a set of (patch, t_start, dt)."""
    lay, f = _lts_case()
    state = ics.to_patches(lay, f)
    g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=1), sched_capacity=1 << 20)
    g.set_state(*state)
    g.advance(t_end=0.002)
    q = Oracle(lay.n, lay.lo, **kw_of(lay, f, time_mode=1, dispatcher=0))
    q.set_state(*state)
    q.advance(t_end=0.002)
    key = lambda s: sorted(zip(*(x.tolist() for x in s)))
    assert key(g.schedule()) == key(q.schedule())
    for a, b in zip(g.get_state(), q.get_state()):
        assert np.array_equal(a, b)


def test_conservation_and_divb_on_gpu():
    lay, f = ics.config_turbulence(seed=5, patches=2, n=16, mach=1.0)
    g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=0))
    g.set_state(*ics.to_patches(lay, f))
    d0 = g.diagnostics()
    g.advance(max_sweeps=10)
    d1 = g.diagnostics()
    U = g.get_state()[0]
    tol = 1e-13 * 10 * np.abs(U).sum() * lay.dx ** 3
    assert abs(d1["mass"] - d0["mass"]) <= tol and abs(d1["energy"] - d0["energy"]) <= tol
    assert np.all(np.abs(d1["mom"] - d0["mom"]) <= tol)
    assert d1["max_divb"] <= 1e-13 * d1["max_b"]


def test_fp32_form_against_fp64():
    """FP32 state and stencil with FP64 times, 20 steps of the linear-wave
    input (amplitude 1e-3) against the FP64 path: relative L1 of the whole
    state <= 1e-5, and, per field, a mean error below 1e-3 of the wave
    amplitude (the transverse field components are pure perturbation, so a
    per-field relative norm would measure FP32 rounding of the O(1)
    background against the 1e-3 wave)."""
    amp = 1e-3
    lay, f = ics.config_linear_waves(amplitude=amp)
    state = ics.to_patches(lay, f)
    g64 = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=0))
    g32 = Dispatch(lay.n, lay.lo, precision=1, **kw_of(lay, f, time_mode=0))
    g64.set_state(*state)
    g32.set_state(*state)
    g64.advance(max_sweeps=20)
    g32.advance(max_sweeps=20)
    a = g64.get_state()
    b = g32.get_state()
    num = sum(np.sum(np.abs(x - y)) for x, y in zip(a, b))
    den = sum(np.sum(np.abs(x)) for x in a)
    assert num / den <= 1e-5
    for x, y in zip(a, b):
        assert np.mean(np.abs(x - y)) <= 1e-3 * amp
    assert np.array_equal(g64.times()[0], g32.times()[0])
    # reported per field: relative L1, and the mean error over the wave
    # amplitude (printed; run with -s to see it)
    cells = np.prod(lay.n, axis=1)
    A, B = split_fields(a, cells), split_fields(b, cells)
    report = {n: {"rel_L1": float(np.abs(x - y).sum() / np.abs(x).sum()),
                  "mean_err_over_amplitude": float(np.mean(np.abs(x - y)) / amp)} for n, x, y in zip(NAMES, A, B)}
    print("FP32_PER_FIELD waves amplitude %g, 20 steps: %s" % (amp, json.dumps(report)))


def test_save_load_resume_is_bit_identical():
    lay, f = _lts_case()
    state = ics.to_patches(lay, f)
    a = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=1))
    a.set_state(*state)
    a.advance(t_end=0.001)
    blob = a.save()
    a.advance(t_end=0.002)
    b = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=1))
    b.load_state(blob)
    b.advance(t_end=0.002)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.times()[0], b.times()[0])


def test_device_pointers_and_fp32_input():
    lay, f = ics.config_linear_waves(n=8, amplitude=1e-3)
    state = ics.to_patches(lay, f)
    g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=0))
    g.set_state(*[torch.from_numpy(x).cuda() for x in state])
    out = [torch.empty(x.size, dtype=torch.float64, device="cuda") for x in state]
    g.get_state(out=out)
    for x, y in zip(out, state):
        assert np.array_equal(x.cpu().numpy(), y)
    g.set_state(*[x.astype(np.float32) for x in state])
    back = g.get_state(dtype=np.float32)
    for x, y in zip(back, state):
        assert np.array_equal(x, y.astype(np.float32))


def test_rejected_inputs():
    lay = ics.cartesian(2, 8)
    base = dict(gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    with pytest.raises(DispatchError) as e:
        Dispatch(lay.n, lay.lo, **base, nguard=8)          # patch not wider than its guard depth
    assert e.value.code == DSP_ERR_INVALID_ARG
    with pytest.raises(DispatchError) as e:
        Dispatch(lay.n, lay.lo, **base, dispatcher=7)
    assert e.value.code in (DSP_ERR_UNSUPPORTED, DSP_ERR_INVALID_ARG)
    with pytest.raises(DispatchError) as e:
        Dispatch(lay.n, lay.lo, **base, dispatcher=0, time_mode=0)   # a global step needs sweeps
    assert e.value.code == DSP_ERR_UNSUPPORTED
    with pytest.raises(DispatchError) as e:
        Dispatch(lay.n[:-1], lay.lo[:-1], **base)           # does not tile the box
    assert e.value.code == DSP_ERR_INVALID_ARG
    f = ics.config_uniform(lay, [1.0, 0, 0, 0, 0.6, 0, 0, 0], 5.0 / 3.0)
    U, bx, by, bz = ics.to_patches(lay, f)
    U[0] = -1.0
    g = Dispatch(lay.n, lay.lo, **base)
    with pytest.raises(DispatchError) as e:
        g.set_state(U, bx, by, bz)
    assert e.value.code == DSP_ERR_UNPHYSICAL


@pytest.mark.parametrize("precision", [0, 1])
def test_ready_queue_dispatcher_matches_sweeps_and_oracle(precision):
    """The persistent ready-queue kernel (blocks claim work, publish patches
    and queue ready neighbours concurrently) gives the same schedule, as a
    set, as the sweep dispatcher and the oracle's time-sorted queue, and the
    same state bit for bit."""
    lay, f = _lts_case()
    state = ics.to_patches(lay, f)
    kw = kw_of(lay, f, time_mode=1)
    q = Dispatch(lay.n, lay.lo, **kw, precision=precision, dispatcher=0, sched_capacity=1 << 20)
    w = Dispatch(lay.n, lay.lo, **kw, precision=precision, dispatcher=1, sched_capacity=1 << 20)
    for g in (q, w):
        g.set_state(*state)
        g.advance(t_end=0.003)
    key = lambda s: sorted(zip(*(x.tolist() for x in s)))
    assert key(q.schedule()) == key(w.schedule())
    for a, b in zip(q.get_state(), w.get_state()):
        assert np.array_equal(a, b)
    assert np.all(q.times()[0] == 0.003)
    if precision == 0:
        o = Oracle(lay.n, lay.lo, **kw_of(lay, f, time_mode=1, dispatcher=0))
        o.set_state(*state)
        o.advance(t_end=0.003)
        assert key(q.schedule()) == key(o.schedule())
        for a, b in zip(q.get_state(), o.get_state()):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_ready_queue_with_mixed_patch_sizes(precision):
    """Patches of 8^3, 16^3 and 32^3 in one ready queue: queue entries carry
    their own tile counts (1 to 16 tiles), claimed tile by tile; the same
    schedule as the sweeps (as a set) and the oracle, states bit for bit."""
    lay, f = _mixed_case(seed=8)
    assert len(np.unique(lay.n[:, 0])) == 3
    state = ics.to_patches(lay, f)
    kw = kw_of(lay, f, time_mode=1)
    q = Dispatch(lay.n, lay.lo, **kw, precision=precision, dispatcher=0, sched_capacity=1 << 20)
    w = Dispatch(lay.n, lay.lo, **kw, precision=precision, dispatcher=1, sched_capacity=1 << 20)
    for g in (q, w):
        g.set_state(*state)
        g.advance(t_end=0.002)
    key = lambda s: sorted(zip(*(x.tolist() for x in s)))
    assert key(q.schedule()) == key(w.schedule())
    for a, b in zip(q.get_state(), w.get_state()):
        assert np.array_equal(a, b)
    if precision == 0:
        o = Oracle(lay.n, lay.lo, **kw_of(lay, f, time_mode=1))
        o.set_state(*state)
        o.advance(t_end=0.002)
        assert key(q.schedule()) == key(o.schedule())
        for a, b in zip(q.get_state(), o.get_state()):
            assert np.array_equal(a, b)


def test_ready_queue_wait_budget_ends_in_timeout_not_a_hang():
    """A wait budget of a few hundred cycles is too short for any update to
    finish: the blocks' waits run out, the kernel returns DSP_ERR_TIMEOUT,
    the context is poisoned and the GPU stays usable."""
    from paper_1705_10774_gb300.dispatch import DSP_ERR_TIMEOUT
    lay, f = _lts_case()
    state = ics.to_patches(lay, f)
    g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=1), dispatcher=0, wait_budget=200)
    g.set_state(*state)
    with pytest.raises(DispatchError) as e:
        g.advance(t_end=0.003)
    assert e.value.code == DSP_ERR_TIMEOUT
    with pytest.raises(DispatchError):
        g.advance(t_end=0.003)          # poisoned
    g.close()
    h = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=1), dispatcher=1)
    h.set_state(*state)
    h.advance(t_end=0.001)              # the device still works


@pytest.mark.parametrize("lts", [False, True])
def test_graph_replay_of_sweeps_is_identical(lts):
    """Sweeps replayed from a captured CUDA graph (batches of 32) give the
    same state and schedule as sweeps launched one by one."""
    if lts:
        lay, f = _lts_case()
        common, run = dict(time_mode=1), dict(t_end=0.003)
    else:
        lay, f = ics.config_linear_waves(n=8, amplitude=1e-3)
        common, run = dict(time_mode=0), dict(max_sweeps=70)
    state = ics.to_patches(lay, f)
    res = []
    for graph in (0, 1):
        g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, **common), graph=graph, sched_capacity=1 << 20)
        g.set_state(*state)
        st = g.advance(**run)
        res.append((g.get_state(), g.schedule(), st))
    (a, sa, _), (b, sb, stb) = res
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    if not lts:
        assert stb["sweeps"] == 70


def _mixed_case(seed=3):
    """A 64^3 box of 2^3 super-blocks of 32^3, each tiled by patches of one
    seeded size out of 8, 16 and 32 cells (tiles are ragged for 8)."""
    lay = ics.mixed_blocks(2, 32, sizes=(8, 16, 32), probs=(1, 1, 1), seed=seed)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    rng = np.random.default_rng(seed)
    v = ics.solenoidal_velocity(shape, lay.box_len, 1.0, 3.0, 1.0, rng)
    A = [ics.gaussian_filtered_noise(shape, lay.box_len, 0.08, rng) * 0.01 for _ in range(3)]
    bx, by, bz = ics.curl_faces(*A, lay.dx)
    rho = np.exp(0.5 * ics.gaussian_filtered_noise(shape, lay.box_len, 0.1, rng))
    f = ics.Fields(rho=rho, v=v, p=np.full(shape, 0.6), bx=bx + 0.5, by=by, bz=bz, gamma=5.0 / 3.0)
    return lay, f


@pytest.mark.parametrize("lts", [False, True])
def test_mixed_patch_sizes(lts):
    """Patches of 8^3, 16^3 and 32^3 side by side: neighbours of different
    sizes supply each other's guard zones through the level map; FP64 stays
    bit-identical to the oracle, schedules equal."""
    lay, f = _mixed_case()
    assert len(np.unique(lay.n[:, 0])) == 3
    if lts:
        common, run = dict(time_mode=1), dict(t_end=0.004)
    else:
        common, run = dict(time_mode=0), dict(max_sweeps=5)
    g, o = pair(lay, f, **common)
    g.advance(**run)
    o.advance(**run)
    assert_same(g, o)
    key = lambda s: sorted(zip(*(x.tolist() for x in s)))
    assert key(g.schedule()) == key(o.schedule())


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_every_kernel_variant_gives_identical_results(precision):
    """The compiled variants of one precision (tile shape, threads per block)
    spread the same arithmetic differently over threads: bit-identical
    states, and the autotuner's choice changes nothing either."""
    import re
    from paper_1705_10774_gb300 import build as B
    ids = [v[0] for v in B.variants() if v[6] == precision and v[7] == 0 and v[8] == 0]
    assert len(ids) >= 2
    lay, f = _mixed_case(seed=4) if precision != 0 else ics.config_linear_waves(n=16, amplitude=1e-3)
    state = ics.to_patches(lay, f)
    outs = []
    for vid in ids + [None]:
        g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=1), precision=precision,
                     variant=-1 if vid is None else vid)
        g.set_state(*state)
        if vid is None:
            chosen, table = g.autotune(reps=1)
            assert chosen in ids and set(table) <= set(ids)
        g.advance(t_end=0.002)
        outs.append(g.get_state())
        g.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_pressure_floor_count_matches_oracle(precision):
    """dsp_stats.floors counts the cells of new slices whose pressure
    recovery took the floor, as the oracle's counter does: every new cell of a
    cold dyadic uniform state (p = 0 exactly, which stays exactly uniform),
    and as many as the oracle on the local-step input."""
    lay = ics.cartesian(2, 8)
    f = ics.config_uniform(lay, [1.0, 0.5, -0.25, 0.125, 0.0, 0.0, 0.0, 0.0], 5.0 / 3.0)
    g, o = pair(lay, f, gpu_extra=dict(precision=precision), time_mode=0)
    st = g.advance(max_sweeps=3)
    o.advance(max_sweeps=3)
    assert st["floors"] == o.stats()["floors"] == st["cell_updates"] == 3 * 8 * 8 ** 3
    if precision == 0:
        lay, f = _lts_case()
        g, o = pair(lay, f, time_mode=1)
        st = g.advance(t_end=0.003)
        o.advance(t_end=0.003)
        assert st["floors"] == o.stats()["floors"]


@pytest.mark.parametrize("precision", [0, 1])
def test_per_size_class_tuning_changes_nothing(precision):
    """Patches of 8^3, 16^3 and 32^3 (three size classes) and of 24^3 next to
    32^3: the autotuner picks a variant and a z run per size class and every
    sweep launches each class's kernel over its part of the work list; the
    states equal an untuned context's bit for bit (and the oracle's in FP64),
    schedules equal, also replayed from CUDA graphs."""
    cases = [_mixed_case(seed=6)]
    lay24 = ics.mixed_blocks(1, 96, sizes=(24, 16), probs=(1, 0), seed=2, remainder=32, rem_size=32)
    X, Y, Z = lay24.base_cells
    rng = np.random.default_rng(2)
    v = ics.solenoidal_velocity((Z, Y, X), lay24.box_len, 1.0, 3.0, 1.0, rng)
    cases.append((lay24, ics.Fields(rho=np.ones((Z, Y, X)), v=v, p=np.full((Z, Y, X), 0.6),
                                    bx=np.full((Z, Y, X), 0.7), by=np.zeros((Z, Y, X)), bz=np.zeros((Z, Y, X)),
                                    gamma=5.0 / 3.0)))
    for lay, f in cases:
        sizes = sorted({tuple(int(x) for x in n) for n in lay.n})
        assert len(sizes) >= 2
        state = ics.to_patches(lay, f)
        outs = []
        for tuned in (False, True):
            g = Dispatch(lay.n, lay.lo, **kw_of(lay, f, time_mode=1), precision=precision, graph=1,
                         sched_capacity=1 << 20)
            g.set_state(*state)
            if tuned:
                g.autotune(reps=1)
                tun = g.tuning()
                assert [tuple(t["size"]) for t in tun] == sizes
                assert {e["cls"] for e in g.tuning_log} == set(range(len(sizes)))
            g.advance(t_end=0.002)
            outs.append((g.get_state(), g.schedule()))
            g.close()
        for a, b in zip(outs[0][0], outs[1][0]):
            assert np.array_equal(a, b)
        key = lambda s: sorted(zip(*(x.tolist() for x in s)))
        assert key(outs[0][1]) == key(outs[1][1])
        if precision == 0:
            o = Oracle(lay.n, lay.lo, **kw_of(lay, f, time_mode=1))
            o.set_state(*state)
            o.advance(t_end=0.002)
            for a, b in zip(outs[1][0], o.get_state()):
                assert np.array_equal(a, b)
