"""GPU parity on two refinement levels (Sec. 3 A: guard values interpolated
in space across a resolution jump): the CUDA path against the FP64 oracle,
which the pins of test_oracle_levels.py tie to prolongation and restriction
identities.  FP64 states are bit-identical (relative L-infinity <= 1e-11),
schedules equal entry by entry."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch
from oracle import Oracle

TOL64 = 1e-11
G53 = 5.0 / 3.0


def smooth_state(lay, seed=7, amp_v=0.5):
    """A smooth seeded state sampled on each patch's own level: log-density
    and velocity from a few random Fourier modes, uniform pressure, faces
    from a random vector potential plus a uniform field."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 3, size=(5, 3))
    ph = rng.random(5) * 2 * np.pi
    mode = lambda i: (lambda x, y, z: np.sin(2 * np.pi * (k[i, 0] * x + k[i, 1] * y + k[i, 2] * z) + ph[i]))
    rho = lambda x, y, z: np.exp(0.3 * mode(0)(x, y, z))
    vel = lambda x, y, z: (amp_v * mode(1)(x, y, z), amp_v * mode(2)(x, y, z), amp_v * mode(3)(x, y, z))
    pre = lambda x, y, z: 0.6 + 0 * x
    A = (lambda x, y, z: 0.02 * mode(4)(x, y, z), lambda x, y, z: 0.02 * mode(0)(y, z, x),
         lambda x, y, z: 0.6 * y + 0.02 * mode(1)(z, x, y))
    return ics.patches_from_functions(lay, rho, vel, pre, G53, potential=A)


def layouts():
    """32^3 level 0 (4^3 patches of 8^3) refined over its central 8^3 cells
    by 2^3 level-1 patches of 8^3; and the same with level 1 over 16^3 cells
    tiled by patches of 16^3 and 8^3 (mixed sizes on level 1)."""
    coarse = ics.cartesian(4, 8)
    a = ics.two_level(coarse, 12, 8, fine_patch=8)
    los, ns = [], []
    for kz in range(2):
        for ky in range(2):
            for kx in range(2):
                o = np.array([kx, ky, kz]) * 16
                if (kx + ky + kz) % 2 == 0:
                    los.append(o)
                    ns.append((16, 16, 16))
                else:
                    for c in np.ndindex(2, 2, 2):
                        los.append(o + 8 * np.array(c))
                        ns.append((8, 8, 8))
    b = ics.two_level(coarse, 8, 16, fine_n=ns, fine_los=los)
    return {"uniform_level1": a, "mixed_level1": b}


def pair(lay, state, **kw):
    common = dict(gamma=G53, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    common.update({k: v for k, v in kw.items() if k in ("time_mode",)})
    gk = {k: v for k, v in kw.items() if k not in ("time_mode",)}
    g = Dispatch(lay.n, lay.lo, level=lay.levels, sched_capacity=1 << 20, **common, **gk)
    g.set_state(*state)
    o = Oracle(lay.n, lay.lo, level=lay.levels, **common)
    o.set_state(*state)
    return g, o


def key(s):
    return sorted(zip(*(x.tolist() for x in s)))


def check_same(g, o, tol=TOL64):
    for name, a, b in zip(("U", "bx", "by", "bz"), g.get_state(), o.get_state()):
        err = float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
        assert err <= tol, (name, err)
    assert np.array_equal(g.times()[0], o.get_times()[0])
    assert key(g.schedule()) == key(o.schedule())


@pytest.mark.parametrize("name", ["uniform_level1", "mixed_level1"])
@pytest.mark.parametrize("time_mode", [0, 1])
def test_two_levels_bit_parity(name, time_mode):
    lay = layouts()[name]
    state = smooth_state(lay)
    g, o = pair(lay, state, time_mode=time_mode)
    run = dict(max_sweeps=6) if time_mode == 0 else dict(t_end=0.01)
    st = g.advance(**run)
    o.advance(**run)
    check_same(g, o)
    if time_mode == 1:
        _, _, dt = g.schedule()
        assert len(np.unique(dt)) >= 2            # the two levels step differently
    assert st["cell_updates"] > 0


def test_two_levels_graph_replay_and_variants_identical():
    """Sweeps replayed from CUDA graphs and every FP64 variant give the same
    two-level state as sweeps launched one by one."""
    from paper_1705_10774_gb300 import build as B
    lay = layouts()["mixed_level1"]
    state = smooth_state(lay, seed=9)
    outs = []
    ids = [v[0] for v in B.variants() if v[6] == 0 and v[7] == 0 and v[8] == 0]
    for graph, variant in [(0, -1), (1, -1)] + [(1, i) for i in ids]:
        g = Dispatch(lay.n, lay.lo, level=lay.levels, gamma=G53, cfl=0.4, base_cells=lay.base_cells,
                     box_len=lay.box_len, time_mode=1, graph=graph, variant=variant)
        g.set_state(*state)
        g.advance(t_end=0.008, max_sweeps=40)
        outs.append(g.get_state())
        g.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)


def test_two_levels_fp32_and_fma_forms():
    """FP32 state within the FP32 tolerance of the FP64 oracle (whole-state
    relative L1 <= 1e-5), FP64 with FMA within 1e-11."""
    lay = layouts()["uniform_level1"]
    state = smooth_state(lay, seed=5)
    o = Oracle(lay.n, lay.lo, level=lay.levels, gamma=G53, cfl=0.4, base_cells=lay.base_cells,
               box_len=lay.box_len, time_mode=1)
    o.set_state(*state)
    o.advance(t_end=0.01)
    ref = o.get_state()
    for prec, tol in ((1, 1e-5), (2, 1e-11)):
        g = Dispatch(lay.n, lay.lo, level=lay.levels, gamma=G53, cfl=0.4, base_cells=lay.base_cells,
                     box_len=lay.box_len, time_mode=1, precision=prec)
        g.set_state(*state)
        g.advance(t_end=0.01)
        out = g.get_state()
        if prec == 1:
            num = sum(float(np.abs(a - b).sum()) for a, b in zip(out, ref))
            den = sum(float(np.abs(b).sum()) for b in ref)
            assert num / den <= tol, num / den
        else:
            for a, b in zip(out, ref):
                assert float(np.max(np.abs(a - b)) / np.max(np.abs(b))) <= tol
        g.close()


def test_two_levels_divb_and_sampled_fill_at_refinement_edges():
    """Every patch keeps zero divergence of its own faces across many local
    steps with two levels (each patch owns all faces of its cells)."""
    lay = layouts()["mixed_level1"]
    state = smooth_state(lay, seed=3)
    g = Dispatch(lay.n, lay.lo, level=lay.levels, gamma=G53, cfl=0.4, base_cells=lay.base_cells,
                 box_len=lay.box_len, time_mode=1)
    g.set_state(*state)
    g.advance(t_end=0.03)
    d = g.diagnostics()
    assert d["max_divb"] <= 1e-13 * d["max_b"], d
