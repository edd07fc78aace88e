"""GPU diagnostics (dsp_diagnostics) against the oracle's, field by field.

The volume integrals of rho, m, E and of the face fields, max |div b| and
max |b| of the newest slices.  The two sides sum the same values in
different orders (the GPU per patch in a strided-then-tree order, the oracle
cell by cell), both with Neumaier-compensated FP64 sums, so each integral must
agree to 1e-13 of the sum of magnitudes of its terms; the maxima are exact.

FP64 (precision 0): after a few steps the two states are bit-identical, so
the diagnostics see the same values.  FP32 (precision 1): the GPU's FP32
state, widened to FP64, is loaded into the oracle, so again both sides see
the same values.  Cases: one level with unequal patch sizes, and two levels
(level-1 cells count with an eighth of the cell volume).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch
from oracle import Oracle

from test_oracle_diagnostics import expected

TOL = 1e-13
NAMES = ["mass", "mom_x", "mom_y", "mom_z", "energy", "bmean_x", "bmean_y", "bmean_z"]


def flat(d):
    return [d["mass"], *d["mom"], d["energy"], *d["bmean"]]


def compare(lay, gd, od, state):
    _, scale, mdiv, mb = expected(lay, state)
    g, o = flat(gd), flat(od)
    for q in range(8):
        assert abs(g[q] - o[q]) <= TOL * scale[q], (NAMES[q], g[q], o[q], scale[q])
    assert gd["max_divb"] == od["max_divb"] == mdiv
    assert gd["max_b"] == od["max_b"] == mb


def _unequal_case():
    lay = ics.cartesian((2, 2, 2), (20, 12, 10), dx=1.0 / 40)
    rng = np.random.default_rng(21)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    v = ics.solenoidal_velocity(shape, lay.box_len, 1.0, 3.0, 1.0, rng)
    A = [ics.gaussian_filtered_noise(shape, lay.box_len, 0.08, rng) * 0.02 for _ in range(3)]
    bx, by, bz = ics.curl_faces(*A, lay.dx)
    f = ics.Fields(rho=1.0 + 0.3 * ics.gaussian_filtered_noise(shape, lay.box_len, 0.1, rng) ** 2, v=v,
                   p=np.full(shape, 0.6), bx=bx + 0.5, by=by + 0.2, bz=bz - 0.1, gamma=5.0 / 3.0)
    return lay, f


def _two_level_case():
    lay = ics.two_level(ics.cartesian(4, 8), 12, 8, fine_patch=8)
    X, Y, Z = lay.base_cells
    rng = np.random.default_rng(5)
    coarse = ics.Layout(n=lay.n[lay.levels == 0], lo=lay.lo[lay.levels == 0], base_cells=lay.base_cells,
                        box_len=lay.box_len)
    shape = (Z, Y, X)
    v = ics.solenoidal_velocity(shape, lay.box_len, 1.0, 2.0, 0.3, rng)
    f = ics.Fields(rho=np.ones(shape), v=v, p=np.full(shape, 0.6), bx=np.full(shape, 0.4),
                   by=np.zeros(shape), bz=np.zeros(shape), gamma=5.0 / 3.0)
    return lay, coarse, f


@pytest.mark.parametrize("precision", [0, 1])
def test_diagnostics_match_oracle_unequal_patches(precision):
    lay, f = _unequal_case()
    state = ics.to_patches(lay, f)
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=0)
    g = Dispatch(lay.n, lay.lo, precision=precision, **kw)
    g.set_state(*state)
    g.advance(max_sweeps=4)
    gd = g.diagnostics()
    if precision == 0:
        o = Oracle(lay.n, lay.lo, **kw)
        o.set_state(*state)
        o.advance(max_sweeps=4)
        now = o.get_state()
        assert all(np.array_equal(a, b) for a, b in zip(g.get_state(), now))
    else:
        now = [a.astype(np.float64) for a in g.get_state(dtype=np.float32)]
        o = Oracle(lay.n, lay.lo, **kw)
        o.set_state(*now)
    compare(lay, gd, o.diagnostics(), now)
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_diagnostics_match_oracle_two_levels(precision):
    lay, coarse, f = _two_level_case()
    base = ics.to_patches(coarse, f)
    # level-1 patches: their parents' values (uniform rho, p, B; the parent's velocity)
    nl0 = coarse.npatch
    parts = []
    for ip in range(lay.npatch):
        nx, ny, nz = (int(a) for a in lay.n[ip])
        if lay.levels[ip] == 0:
            continue
        lo = lay.lo[ip] // 2
        v = [f.v[d][lo[2]:lo[2] + nz // 2, lo[1]:lo[1] + ny // 2, lo[0]:lo[0] + nx // 2]
             .repeat(2, 0).repeat(2, 1).repeat(2, 2) for d in range(3)]
        c = nx * ny * nz
        rho = np.ones(c)
        E = 0.6 / (f.gamma - 1) + 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2).ravel() + 0.5 * 0.4 ** 2
        u = np.concatenate([rho, v[0].ravel(), v[1].ravel(), v[2].ravel(), E])
        parts.append((u, np.full((nx + 1) * ny * nz, 0.4), np.zeros(nx * (ny + 1) * nz), np.zeros(nx * ny * (nz + 1))))
    state = [np.concatenate([base[k]] + [p_[k] for p_ in parts]) for k in range(4)]
    assert int((lay.levels[:nl0] == 0).sum()) == nl0
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1)
    g = Dispatch(lay.n, lay.lo, level=lay.levels, precision=precision, **kw)
    g.set_state(*state)
    g.advance(max_sweeps=3)
    gd = g.diagnostics()
    if precision == 0:
        o = Oracle(lay.n, lay.lo, level=lay.levels, **kw)
        o.set_state(*state)
        o.advance(max_sweeps=3)
        now = o.get_state()
        assert all(np.array_equal(a, b) for a, b in zip(g.get_state(), now))
    else:
        now = [a.astype(np.float64) for a in g.get_state(dtype=np.float32)]
        o = Oracle(lay.n, lay.lo, level=lay.levels, **kw)
        o.set_state(*now)
    compare(lay, gd, o.diagnostics(), now)
    g.close()
