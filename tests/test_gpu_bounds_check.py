"""The bounds-checked build (libdispatch_gpu_checked.so, -DDSP_BOUNDS_CHECK):
every global load and store of the update kernel is tested against the
slab of slices and the cross-level guard buffers, and an address outside
them would end the run with DSP_ERR_BOUNDS instead of a fault.  On small
cases that reach every gather path -- ragged tiles and z runs, a patch that
is its own neighbour, mixed patch sizes, two levels with cross-level guard
buffers, local steps with time interpolation -- the checked build must run
clean and give the regular build's results bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch

from test_gpu_parity import _lts_case, _mixed_case


def cases():
    out = []
    lay = ics.cartesian((2, 2, 2), (20, 12, 10), dx=1.0 / 40)
    X, Y, Z = lay.base_cells
    rng = np.random.default_rng(9)
    v = ics.solenoidal_velocity((Z, Y, X), lay.box_len, 1.0, 3.0, 1.0, rng)
    out.append(("ragged", lay, ics.Fields(rho=np.ones((Z, Y, X)), v=v, p=np.full((Z, Y, X), 0.6),
                                          bx=np.full((Z, Y, X), 0.5), by=np.zeros((Z, Y, X)),
                                          bz=np.zeros((Z, Y, X)), gamma=5.0 / 3.0), dict(tile_z=3, time_mode=0)))
    lay = ics.cartesian(1, 8)
    out.append(("self", lay, ics.config_uniform(lay, [1.0, 0.2, -0.1, 0.3, 0.6, 0.8, 0.1, -0.2], 5.0 / 3.0, seed=4,
                                                eps=1e-3), dict(time_mode=0)))
    lay, f = _mixed_case(seed=7)
    out.append(("mixed", lay, f, dict(time_mode=1)))
    lay, f = _lts_case()
    out.append(("lts", lay, f, dict(time_mode=1)))
    return out


def two_level_case():
    lay = ics.two_level(ics.cartesian(4, 8), 12, 8, fine_patch=8)
    rng = np.random.default_rng(3)
    parts = []
    for nx, ny, nz in lay.n.astype(int):
        c = nx * ny * nz
        u = np.concatenate([1.0 + 0.1 * rng.random(c), 0.1 * rng.standard_normal(3 * c), 2.0 + 0.1 * rng.random(c)])
        parts.append((u, np.full((nx + 1) * ny * nz, 0.3), np.zeros(nx * (ny + 1) * nz), np.zeros(nx * ny * (nz + 1))))
    return lay, [np.concatenate([p_[k] for p_ in parts]) for k in range(4)]


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_checked_build_runs_clean_and_matches(precision):
    for name, lay, f, kw in cases():
        state = ics.to_patches(lay, f)
        res = []
        for checked in (False, True):
            g = Dispatch(lay.n, lay.lo, gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                         precision=precision, checked=checked, **kw)
            g.set_state(*state)
            st = g.advance(t_end=0.002) if kw.get("time_mode") == 1 else g.advance(max_sweeps=4)
            assert st["status"] == 0, name
            res.append(g.get_state())
            g.close()
        for a, b in zip(*res):
            assert np.array_equal(a, b), name
    lay, state = two_level_case()
    res = []
    for checked in (False, True):
        g = Dispatch(lay.n, lay.lo, level=lay.levels, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells,
                     box_len=lay.box_len, precision=precision, time_mode=1, checked=checked)
        g.set_state(*state)
        assert g.advance(t_end=0.002)["status"] == 0
        res.append(g.get_state())
        g.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)
