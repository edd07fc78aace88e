"""GPU parity of readiness with grace and of the time inter- and
extrapolation order (DISPATCH I, Sec. 3 B: Eq. 1 with g > 0, linear or
quadratic time inter- and extrapolation of guard values): the CUDA path
against the FP64 oracle, whose choice of slices, weights, grace limit and
kept-slice rule test_oracle_time.py pins.  FP64 without FMA: states
bit-identical, schedules equal entry by entry."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch, DispatchError, DSP_ERR_INVALID_ARG, DSP_ERR_UNSUPPORTED
from oracle import Oracle


def lts_case():
    """512 patches of 4^3 with steps spanning a factor > 200 (log-normal
    density, a hot sphere)."""
    return ics.config_lts(patches=8, n=4, sigma_ln=2.0, hot_radius=0.2, hot_factor=300.0)


def pair(lay, state, gamma, run, levels=None, gpu_extra=None, **common):
    lv = {} if levels is None else dict(level=levels)
    base = dict(gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1, **common)
    g = Dispatch(lay.n, lay.lo, **lv, **base, sched_capacity=1 << 21, **(gpu_extra or {}))
    g.set_state(*state)
    o = Oracle(lay.n, lay.lo, **lv, **base)
    o.set_state(*state)
    g.advance(**run)
    o.advance(**run)
    return g, o


def assert_bit_identical(g, o, as_set=False):
    for name, a, b in zip(("U", "bx", "by", "bz"), g.get_state(), o.get_state()):
        assert np.array_equal(a, b), (name, float(np.max(np.abs(a - b))))
    assert np.array_equal(g.times()[0], o.get_times()[0])
    if as_set:
        key = lambda s: sorted(zip(*(x.tolist() for x in s)))
        assert key(g.schedule()) == key(o.schedule())
    else:
        for x, y in zip(g.schedule(), o.schedule()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("grace,order,ns", [(0.6, 1, 3), (0.0, 2, 3), (0.6, 2, 4), (0.3, 1, 5)])
def test_grace_and_time_order_bit_parity(grace, order, ns):
    """Local steps with grace (guard values extrapolated where a patch runs
    ahead of a neighbour) and with quadratic time interpolation through
    three slices, with three to five slices per patch."""
    lay, f = lts_case()
    g, o = pair(lay, ics.to_patches(lay, f), f.gamma, dict(t_end=0.002), grace=grace, time_order=order,
                nslices=ns)
    assert_bit_identical(g, o)


def test_quadratic_time_interpolation_across_levels():
    """Two levels: level-1 guard values prolonged from level-0 slices
    interpolated quadratically in time (level-1 steps are half the level-0
    steps, so every other level-1 step falls between level-0 slices)."""
    from test_gpu_levels import layouts, smooth_state
    lay = layouts()["mixed_level1"]
    g, o = pair(lay, smooth_state(lay), 5.0 / 3.0, dict(t_end=0.01), levels=lay.levels, time_order=2)
    assert_bit_identical(g, o, as_set=True)


def test_fp32_and_graph_replay_with_grace_and_quadratic_order():
    """Sweeps replayed from CUDA graphs give the state of sweeps launched one
    by one; the FP32 form stays within 1e-5 relative L1 of the FP64 one."""
    lay, f = lts_case()
    st = ics.to_patches(lay, f)
    base = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1, grace=0.6,
                time_order=2, nslices=4)
    outs = []
    for extra in (dict(graph=0), dict(graph=1), dict(precision=1)):
        g = Dispatch(lay.n, lay.lo, **base, **extra)
        g.set_state(*st)
        g.advance(t_end=0.002)
        outs.append(g.get_state())
        g.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    num = sum(float(np.abs(a - b).sum()) for a, b in zip(outs[0], outs[2]))
    den = sum(float(np.abs(a).sum()) for a in outs[0])
    assert num / den <= 1e-5, num / den


def test_time_parameters_are_rejected():
    lay, f = ics.config_linear_waves(n=8, amplitude=1e-3)
    base = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1)
    for bad, code in ((dict(grace=1.0), DSP_ERR_INVALID_ARG), (dict(grace=-0.5), DSP_ERR_INVALID_ARG),
                      (dict(time_order=3), DSP_ERR_INVALID_ARG), (dict(nslices=17), DSP_ERR_INVALID_ARG),
                      (dict(grace=0.3, time_order=2, nslices=3), DSP_ERR_INVALID_ARG),
                      (dict(grace=0.3, dispatcher=0), DSP_ERR_UNSUPPORTED)):
        with pytest.raises(DispatchError) as e:
            Dispatch(lay.n, lay.lo, **base, **bad)
        assert e.value.code == code, bad
