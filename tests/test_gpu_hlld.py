"""GPU parity of the HLLD face flux (Miyoshi & Kusano 2005; the MHD solver of
Sec. 5.3's cost comparison): the CUDA path with riemann = 1 against the FP64
oracle with riemann = 1, whose HLLD is pinned in test_oracle_hlld.py (exact
contacts and rotational discontinuities, integral consistency of the fan).

FP64 without FMA (precision 0) evaluates the oracle's operation sequence, so
the states must be bit-identical and the schedules equal entry by entry; the
FMA form (precision 2) stays within 1e-11, FP32 within 1e-5 relative L1."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import build as B
from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch, DispatchError, DSP_ERR_INVALID_ARG
from oracle import Oracle

HLLD = 1


def kw_of(lay, gamma, **extra):
    d = dict(gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    d.update(extra)
    return d


def key(s):
    return sorted(zip(*(x.tolist() for x in s)))


def run_pair(lay, state, gamma, run, gpu_extra=None, levels=None, **common):
    lv = {} if levels is None else dict(level=levels)
    g = Dispatch(lay.n, lay.lo, **lv, **kw_of(lay, gamma, **common), riemann=HLLD, sched_capacity=1 << 20,
                 **(gpu_extra or {}))
    g.set_state(*state)
    o = Oracle(lay.n, lay.lo, **lv, **kw_of(lay, gamma, **common), riemann=HLLD)
    o.set_state(*state)
    st = g.advance(**run)
    o.advance(**run)
    return g, o, st


def assert_bit_identical(g, o, queue=False):
    for name, a, b in zip(("U", "bx", "by", "bz"), g.get_state(), o.get_state()):
        assert np.array_equal(a, b), (name, float(np.max(np.abs(a - b))))
    assert np.array_equal(g.times()[0], o.get_times()[0])
    if queue:
        assert key(g.schedule()) == key(o.schedule())
    else:
        for x, y in zip(g.schedule(), o.schedule()):
            assert np.array_equal(x, y)


def brio_wu(axis, bn, n=64, thin=4):
    """A Brio-Wu tube (rho, p) = (1, 1) | (0.125, 0.1), tangential field
    +1 | -1 along the next axis, normal field bn, gamma = 2, on a periodic box
    of `n` cells along `axis` in four patches (two interfaces)."""
    cpp = [thin, thin, thin]
    cpp[axis] = n // 4
    ppa = [1, 1, 1]
    ppa[axis] = 4
    lay = ics.cartesian(ppa, cpp, dx=1.0 / n)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    c = (np.arange(lay.base_cells[axis]) + 0.5) / n
    s = [1, 1, 1]
    s[2 - axis] = -1
    left = np.broadcast_to(((c >= 0.25) & (c < 0.75)).reshape(s), shape)
    b = [np.zeros(shape) for _ in range(3)]
    b[axis][...] = bn
    b[(axis + 1) % 3][...] = np.where(left, 1.0, -1.0)     # varies along `axis` only: zero divergence
    f = ics.Fields(rho=np.where(left, 1.0, 0.125), v=np.zeros((3,) + shape), p=np.where(left, 1.0, 0.1),
                   bx=b[0], by=b[1], bz=b[2], gamma=2.0)
    return lay, f


def test_hlld_linear_waves_bit_parity():
    """Eight 16^3 patches, four seeded linear modes, 20 global steps."""
    lay, f = ics.config_linear_waves()
    g, o, st = run_pair(lay, ics.to_patches(lay, f), f.gamma, dict(max_sweeps=20), time_mode=0)
    assert st["patch_updates"] == 160
    assert_bit_identical(g, o)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("bn", [0.75, 0.0])
def test_hlld_brio_wu_tubes_bit_parity(axis, bn):
    """Shock tubes along each axis, with and without a normal field: every
    region of the HLLD fan is taken (outer states, the four star states),
    and with bn = 0 the double-star states collapse onto the star ones.  The
    HLLD result also differs from the HLL one (the flag reaches the kernel)."""
    lay, f = brio_wu(axis, bn)
    state = ics.to_patches(lay, f)
    g, o, _ = run_pair(lay, state, f.gamma, dict(max_sweeps=30), time_mode=0)
    assert_bit_identical(g, o)
    h = Dispatch(lay.n, lay.lo, **kw_of(lay, f.gamma, time_mode=0), riemann=0)
    h.set_state(*state)
    h.advance(max_sweeps=30)
    assert not np.array_equal(h.get_state()[0], g.get_state()[0])


def test_hlld_field_aligned_blob_takes_the_degenerate_branch():
    """A dense blob in a strong field along x (Alfven speed 2 above the sound
    speed 0.45): away from the blob the x-faces see S_L = u - c_A, so the
    star-state denominator vanishes to round-off and the degenerate branch
    (tangential velocity and field of the side kept) is taken; inside, the
    regular one.  Bit parity over local steps."""
    lay = ics.cartesian(2, 12)
    rho = lambda x, y, z: 1.0 + 2.0 * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) / 0.02)
    vel = lambda x, y, z: (0.3 + 0 * x, 0.1 * np.sin(2 * np.pi * y) + 0 * x, 0 * x)
    pre = lambda x, y, z: 0.12 + 0 * x
    faces = (lambda x, y, z: 2.0 + 0 * x, lambda x, y, z: 0 * x, lambda x, y, z: 0 * x)
    state = ics.patches_from_functions(lay, rho, vel, pre, 5.0 / 3.0, faces=faces)
    g, o, _ = run_pair(lay, state, 5.0 / 3.0, dict(t_end=0.02), time_mode=1)
    assert_bit_identical(g, o)


def _lts_case():
    return ics.config_lts(patches=6, n=4, sigma_ln=1.0, hot_radius=0.15, hot_factor=100.0)


@pytest.mark.parametrize("dispatcher", [1, 0])
def test_hlld_local_steps_sweeps_and_queue(dispatcher):
    """Local steps spanning a factor > 8 under the sweep dispatcher (schedule
    equal entry by entry) and the persistent ready-queue kernel (schedule
    equal as a set): states bit-identical to the oracle's."""
    lay, f = _lts_case()
    g, o, _ = run_pair(lay, ics.to_patches(lay, f), f.gamma, dict(t_end=0.003),
                       gpu_extra=dict(dispatcher=dispatcher), time_mode=1)
    assert len(np.unique(o.schedule()[2])) >= 3
    assert_bit_identical(g, o, queue=dispatcher == 0)


def test_hlld_turbulence_with_graph_replay():
    """A Mach-2 turbulent 32^3 box (2^3 patches of 16^3): sweeps replayed
    from CUDA graphs, bit-identical to the oracle."""
    lay, f = ics.config_turbulence(seed=5, patches=2, n=16, mach=2.0)
    g, o, _ = run_pair(lay, ics.to_patches(lay, f), f.gamma, dict(t_end=0.01),
                       gpu_extra=dict(graph=1), time_mode=1)
    assert_bit_identical(g, o)


@pytest.mark.parametrize("time_mode", [0, 1])
def test_hlld_two_levels_bit_parity(time_mode):
    """Two refinement levels (level 1 over the central 8^3 of a 32^3 level 0)
    with HLLD fluxes: guard values prolonged and restricted across the jump."""
    from test_gpu_levels import layouts, smooth_state
    lay = layouts()["uniform_level1"]
    run = dict(max_sweeps=6) if time_mode == 0 else dict(t_end=0.01)
    g, o, _ = run_pair(lay, smooth_state(lay), 5.0 / 3.0, run, levels=lay.levels, time_mode=time_mode)
    assert_bit_identical(g, o, queue=True)


def test_hlld_fma_and_fp32_forms():
    """FP64 with FMA within 1e-11 of the oracle (whole-state relative
    L-infinity, the linear-wave input being a 1e-6 perturbation); FP32 state
    within 1e-5 relative L1 of the FP64 HLLD path on a 1e-3 wave."""
    lay, f = ics.config_linear_waves()
    state = ics.to_patches(lay, f)
    g, o, _ = run_pair(lay, state, f.gamma, dict(max_sweeps=20), gpu_extra=dict(precision=2), time_mode=0)
    out, ref = g.get_state(), o.get_state()
    num = max(float(np.max(np.abs(a - b))) for a, b in zip(out, ref))
    den = max(float(np.max(np.abs(b))) for b in ref)
    assert num / den <= 1e-11, num / den

    lay, f = ics.config_linear_waves(amplitude=1e-3)
    state = ics.to_patches(lay, f)
    outs = []
    for prec in (0, 1):
        h = Dispatch(lay.n, lay.lo, **kw_of(lay, f.gamma, time_mode=0), precision=prec, riemann=HLLD)
        h.set_state(*state)
        h.advance(max_sweeps=20)
        outs.append(h.get_state())
    num = sum(float(np.abs(a - b).sum()) for a, b in zip(*outs))
    den = sum(float(np.abs(a).sum()) for a in outs[0])
    assert num / den <= 1e-5, num / den


def test_hlld_variant_selection():
    """The autotuner picks among the HLLD variants only; an HLL variant id
    or an unknown solver is rejected."""
    lay, f = ics.config_linear_waves(n=8, amplitude=1e-3)
    state = ics.to_patches(lay, f)
    hlld_ids = [v[0] for v in B.variants() if v[6] == 0 and v[7] == HLLD and v[8] == 0]
    hll_ids = [v[0] for v in B.variants() if v[6] == 0 and v[7] == 0 and v[8] == 0]
    g = Dispatch(lay.n, lay.lo, **kw_of(lay, f.gamma, time_mode=1), riemann=HLLD)
    g.set_state(*state)
    chosen, table = g.autotune(reps=1)
    assert chosen in hlld_ids and set(table) <= set(hlld_ids)
    g.close()
    with pytest.raises(DispatchError) as e:
        Dispatch(lay.n, lay.lo, **kw_of(lay, f.gamma), riemann=HLLD, variant=hll_ids[0])
    assert e.value.code == DSP_ERR_INVALID_ARG
    with pytest.raises(DispatchError) as e:
        Dispatch(lay.n, lay.lo, **kw_of(lay, f.gamma), riemann=2)
    assert e.value.code == DSP_ERR_INVALID_ARG

