"""GPU parity of the non-ideal MHD terms (DISPATCH I, Sec. 4.3: Ohmic
E = eta J, ambipolar E = -v_D x B, their Poynting flux and step limits):
the CUDA path against the FP64 oracle with the same terms, whose non-ideal
arithmetic test_oracle_nonideal.py pins (Table 1's C-shocks, Beltrami-field
decay and steadiness, damped Alfven waves, conservation, step limits).

FP64 without FMA (precision 0) evaluates the oracle's operation sequence:
states bit-identical, schedules equal entry by entry (sweeps) or as sets
(ready queue).  FP64 with FMA within 1e-11, FP32 within 1e-5 relative L1."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import build as B
from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch, DispatchError, DSP_ERR_INVALID_ARG
from oracle import Oracle

G53 = 5.0 / 3.0
BOTH = dict(eta=0.01, gamma_ad=50.0, rho_i=0.7)


def key(s):
    return sorted(zip(*(x.tolist() for x in s)))


def run_pair(lay, state, gamma, run, ni, gpu_extra=None, levels=None, **common):
    lv = {} if levels is None else dict(level=levels)
    base = dict(gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, **common)
    g = Dispatch(lay.n, lay.lo, **lv, **base, **ni, sched_capacity=1 << 20, **(gpu_extra or {}))
    g.set_state(*state)
    o = Oracle(lay.n, lay.lo, **lv, **base, **ni)
    o.set_state(*state)
    st = g.advance(**run)
    o.advance(**run)
    return g, o, st


def assert_bit_identical(g, o, as_set=False):
    for name, a, b in zip(("U", "bx", "by", "bz"), g.get_state(), o.get_state()):
        assert np.array_equal(a, b), (name, float(np.max(np.abs(a - b))))
    assert np.array_equal(g.times()[0], o.get_times()[0])
    if as_set:
        assert key(g.schedule()) == key(o.schedule())
    else:
        for x, y in zip(g.schedule(), o.schedule()):
            assert np.array_equal(x, y)


def turbulent(patches=2, n=16, seed=5):
    lay, f = ics.config_turbulence(seed=seed, patches=patches, n=n, mach=1.0)
    return lay, ics.to_patches(lay, f), f.gamma


@pytest.mark.parametrize("ni", [dict(eta=0.02), dict(gamma_ad=20.0, rho_i=1.0), BOTH],
                         ids=["ohmic", "ambipolar", "both"])
@pytest.mark.parametrize("time_mode", [0, 1])
def test_nonideal_turbulence_bit_parity(ni, time_mode):
    """A Mach-1 turbulent 32^3 box (2^3 patches of 16^3) with each term
    alone and both: states bit-identical to the oracle after several steps,
    under global and local steps."""
    lay, st, gamma = turbulent()
    run = dict(max_sweeps=6) if time_mode == 0 else dict(t_end=0.004)
    g, o, stats = run_pair(lay, st, gamma, run, ni, time_mode=time_mode)
    assert stats["cell_updates"] > 0
    assert_bit_identical(g, o)


def test_nonideal_ragged_tiles_and_non_cubic_patches():
    """Patches of 20 x 10 x 6 cells: x spans a full and a partial 16-wide
    tile, y two full and a partial 4-high FP64 tile, z runs of 6."""
    lay = ics.cartesian((2, 2, 2), (20, 10, 6), dx=1.0 / 40)
    rng = np.random.default_rng(11)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    v = ics.solenoidal_velocity(shape, lay.box_len, 1.0, 3.0, 0.8, rng)
    A = [ics.gaussian_filtered_noise(shape, lay.box_len, 0.08, rng) * 0.02 for _ in range(3)]
    bx, by, bz = ics.curl_faces(*A, lay.dx)
    f = ics.Fields(rho=1.0 + 0.3 * ics.gaussian_filtered_noise(shape, lay.box_len, 0.1, rng) ** 2, v=v,
                   p=np.full(shape, 0.6), bx=bx + 0.5, by=by + 0.2, bz=bz, gamma=G53)
    g, o, _ = run_pair(lay, ics.to_patches(lay, f), G53, dict(t_end=0.003), BOTH, time_mode=1,
                       gpu_extra=dict(tile_z=4))
    assert_bit_identical(g, o)


def test_nonideal_cshock_bit_parity():
    """The steady non-isothermal ambipolar C-shock of Table 1 (five patches
    of 30 x 4 x 4) and the Ohmic one: bit-identical to the oracle over local
    steps."""
    from test_oracle_nonideal import cshock_setup
    for name in ("ad_noniso", "ohm"):
        lay, f, gamma, kw, *_ = cshock_setup(name, 150)
        g, o, _ = run_pair(lay, ics.to_patches(lay, f), gamma, dict(t_end=0.01), kw, time_mode=1)
        assert_bit_identical(g, o)


def test_nonideal_ready_queue_and_graph_replay():
    """The persistent ready-queue kernel (schedule equal as a set) and sweeps
    replayed from CUDA graphs: bit-identical to the oracle."""
    lay, f = ics.config_lts(patches=4, n=8, sigma_ln=1.0, hot_radius=0.15, hot_factor=20.0)
    st = ics.to_patches(lay, f)
    for extra, as_set in ((dict(dispatcher=0), True), (dict(graph=1), False)):
        g, o, _ = run_pair(lay, st, f.gamma, dict(t_end=0.002), BOTH, time_mode=1, gpu_extra=extra)
        assert_bit_identical(g, o, as_set=as_set)


def test_nonideal_two_levels_bit_parity():
    """Two refinement levels (level 1 over the central 8^3 of a 32^3 level 0):
    the currents use each level's own cell size."""
    from test_gpu_levels import layouts, smooth_state
    lay = layouts()["uniform_level1"]
    g, o, _ = run_pair(lay, smooth_state(lay), G53, dict(t_end=0.005), BOTH, levels=lay.levels, time_mode=1)
    assert_bit_identical(g, o, as_set=True)


def test_nonideal_fma_and_fp32_forms():
    """FP64 with FMA within 1e-11 of the oracle; FP32 within 1e-5 relative L1
    of the FP64 path; conservation and div B on the GPU."""
    lay, st, gamma = turbulent()
    g, o, _ = run_pair(lay, st, gamma, dict(t_end=0.004), BOTH, time_mode=1, gpu_extra=dict(precision=2))
    for a, b in zip(g.get_state(), o.get_state()):
        assert float(np.max(np.abs(a - b)) / np.max(np.abs(b))) <= 1e-11
    outs = []
    for prec in (0, 1):
        h = Dispatch(lay.n, lay.lo, gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                     time_mode=0, precision=prec, **BOTH)
        h.set_state(*st)
        d0 = h.diagnostics()
        h.advance(max_sweeps=8)
        d1 = h.diagnostics()
        outs.append(h.get_state())
        if prec == 0:
            U = outs[-1][0]
            tol = 1e-13 * 8 * np.abs(U).sum() * lay.dx ** 3
            assert abs(d1["mass"] - d0["mass"]) <= tol and abs(d1["energy"] - d0["energy"]) <= tol
            assert d1["max_divb"] <= 1e-13 * d1["max_b"]
    num = sum(float(np.abs(a - b).sum()) for a, b in zip(*outs))
    den = sum(float(np.abs(a).sum()) for a in outs[0])
    assert num / den <= 1e-5, num / den


def test_nonideal_variant_selection_and_rejected_parameters():
    """Non-ideal contexts run the non-ideal variants only (the autotuner
    included); an ideal variant id with non-ideal terms, a negative
    coefficient or an ambipolar term without ion density is rejected."""
    lay, st, gamma = turbulent(n=8)
    base = dict(gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1)
    ni_ids = [v[0] for v in B.variants() if v[6] == 0 and v[7] == 0 and v[8] == 1]
    ideal_ids = [v[0] for v in B.variants() if v[6] == 0 and v[7] == 0 and v[8] == 0]
    g = Dispatch(lay.n, lay.lo, **base, **BOTH)
    g.set_state(*st)
    chosen, table = g.autotune(reps=1)
    assert chosen in ni_ids and set(table) <= set(ni_ids)
    g.close()
    for bad in (dict(eta=0.01, variant=ideal_ids[0]), dict(eta=-1.0), dict(gamma_ad=5.0, rho_i=0.0),
                dict(gamma_ad=-1.0), dict(eta=0.01, c_ohm=-0.1)):
        with pytest.raises(DispatchError) as e:
            Dispatch(lay.n, lay.lo, **base, **bad)
        assert e.value.code == DSP_ERR_INVALID_ARG


def test_nonideal_with_hlld_faces():
    """HLLD face fluxes together with both non-ideal terms: bit-identical to
    the oracle with the same options (FP64 exact), FMA within 1e-11."""
    lay, st, gamma = turbulent()
    for prec in (0, 2):
        base = dict(gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1, riemann=1,
                    **BOTH)
        g = Dispatch(lay.n, lay.lo, **base, precision=prec, sched_capacity=1 << 20)
        g.set_state(*st)
        o = Oracle(lay.n, lay.lo, **base)
        o.set_state(*st)
        g.advance(t_end=0.004)
        o.advance(t_end=0.004)
        if prec == 0:
            assert_bit_identical(g, o)
        else:
            for a, b in zip(g.get_state(), o.get_state()):
                assert float(np.max(np.abs(a - b)) / np.max(np.abs(b))) <= 1e-11


@pytest.mark.parametrize("name,t_end,bound,ratio", [("ad_iso", 0.2, 0.01, 2.0), ("ad_noniso", 0.2, 0.015, 2.0),
                                                     ("ohm", 0.3, 0.03, 1.0)])
def test_cshock_jump_settles_to_steady_profile_on_gpu(name, t_end, bound, ratio):
    """Sec. 5.4's three C-shock experiments on the GPU (FP64 without FMA,
    local steps, CUDA graphs), from the Table 1 discontinuity on a periodic
    box of 4 (300 cells, patches of 30 x 4 x 4): B_y settles to the steady
    C-shock profile of the conservation laws (mean distance within 0.3 of
    the shock, over the jump, below `bound`), and the patch steps differ by
    a factor of 2 in the ambipolar runs and not at all in the Ohmic one, as
    the paper reports.  The figures are printed (run with -s)."""
    import json
    import time
    from cshock_ode import jump_input, most_common_steps, profile_error
    lay, f, gamma, kw, xc = jump_input(name)
    g = Dispatch(lay.n, lay.lo, gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                 time_mode=1, graph=1, precision=0, sched_capacity=1 << 22, **kw)
    g.set_state(*ics.to_patches(lay, f))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = g.advance(t_end=t_end)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    By = ics.from_patches(lay, *g.get_state())[2][0, 0]
    steps = most_common_steps(g.schedule(), lay.npatch)
    err = profile_error(name, xc, By, 3.0)
    r = float(steps.max() / steps.min())
    print("CSHOCK %s" % json.dumps({"case": name, "t_end": t_end, "profile_error": err, "step_ratio": r,
                                    "patch_updates": st["patch_updates"], "seconds": el}))
    g.close()
    assert err < bound, err
    assert r == ratio, r


@pytest.mark.parametrize("precision", [0, 2])
def test_nonideal_variants_identical(precision):
    """The non-ideal variants of one precision (threads per block) give
    bit-identical states with both terms on, the autotuner's choice
    included."""
    ids = [v[0] for v in B.variants() if v[6] == precision and v[7] == 0 and v[8] == 1]
    assert len(ids) >= 2
    lay, st, gamma = turbulent()
    base = dict(gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1)
    outs = []
    for vid in ids + [None]:
        g = Dispatch(lay.n, lay.lo, **base, **BOTH, precision=precision, variant=-1 if vid is None else vid)
        g.set_state(*st)
        if vid is None:
            chosen, table = g.autotune(reps=1)
            assert chosen in ids and set(table) <= set(ids)
        g.advance(t_end=0.004)
        outs.append(g.get_state())
        g.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)
