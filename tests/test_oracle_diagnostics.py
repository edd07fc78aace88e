"""Pins of the oracle's diagnostics (the conservation sums and div B that
the conservation tests and the FP32 drift figures rest on).

What is pinned, each independently of the oracle's own loops:
  - the volume integrals of rho, m and E against exact (math.fsum) sums of
    numpy reshapes of the same patch arrays, times each patch's own cell
    volume, on patches of unequal sizes along the three axes;
  - the face-field integrals against exact sums over the low face of every
    cell (numpy slices that drop each patch's upper boundary face);
  - max |div b| against np.diff of the reshaped face arrays, and a planted
    jump on a single face of each orientation (interior faces, and a
    patch's upper boundary face, which only the last cell's divergence
    sees) must come out exactly;
  - max |b| over the low faces of every cell, which for a periodic state
    cut from one global field is the maximum over all stored faces;
  - closed forms: a uniform state integrates to its value times the box
    volume; with a second level at half the cell size, level-1 cells count
    with dx^3/8 and the level-0 cells under them still count, so the total
    is the value times (box volume + refined volume).
"""
import math

import numpy as np
import pytest

from paper_1705_10774_gb300 import ics
from oracle import Oracle


def _split(lay, U, bx, by, bz):
    """Per patch: U (5, nz, ny, nx), bx (nz, ny, nx+1), by (nz, ny+1, nx),
    bz (nz+1, ny, nx)."""
    out, oU, ox, oy, oz = [], 0, 0, 0, 0
    for nx, ny, nz in lay.n.astype(int):
        c = nx * ny * nz
        u = U[oU:oU + 5 * c].reshape(5, nz, ny, nx)
        fx = bx[ox:ox + (nx + 1) * ny * nz].reshape(nz, ny, nx + 1)
        fy = by[oy:oy + nx * (ny + 1) * nz].reshape(nz, ny + 1, nx)
        fz = bz[oz:oz + nx * ny * (nz + 1)].reshape(nz + 1, ny, nx)
        out.append((u, fx, fy, fz))
        oU += 5 * c
        ox += (nx + 1) * ny * nz
        oy += nx * (ny + 1) * nz
        oz += nx * ny * (nz + 1)
    return out


def expected(lay, state):
    """The diagnostics written with numpy reductions and exact sums."""
    dx = lay.dx
    lev = lay.levels
    parts = _split(lay, *state)
    sums = [[] for _ in range(8)]
    mdiv, mb = 0.0, 0.0
    for ip, (u, fx, fy, fz) in enumerate(parts):
        dV = (dx / 2 ** int(lev[ip])) ** 3
        for q in range(5):
            sums[q].extend((u[q] * dV).ravel().tolist())
        sums[5].extend((fx[:, :, :-1] * dV).ravel().tolist())
        sums[6].extend((fy[:, :-1, :] * dV).ravel().tolist())
        sums[7].extend((fz[:-1, :, :] * dV).ravel().tolist())
        div = np.diff(fx, axis=2) + np.diff(fy, axis=1) + np.diff(fz, axis=0)
        mdiv = max(mdiv, float(np.max(np.abs(div))))
        mb = max(mb, float(np.max(np.abs(fx[:, :, :-1]))), float(np.max(np.abs(fy[:, :-1, :]))),
                 float(np.max(np.abs(fz[:-1, :, :]))))
    tot = [math.fsum(s) for s in sums]
    scale = [math.fsum(abs(x) for x in s) for s in sums]
    return tot, scale, mdiv, mb


def oracle_diag(lay, state, gamma=5.0 / 3.0):
    o = Oracle(lay.n, lay.lo, level=lay.level, gamma=gamma, cfl=0.4, base_cells=lay.base_cells,
               box_len=lay.box_len)
    o.set_state(*state)
    d = o.diagnostics()
    return [d["mass"], *d["mom"], d["energy"], *d["bmean"]], d["max_divb"], d["max_b"]


def _random_state(lay, seed):
    rng = np.random.default_rng(seed)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    v = ics.solenoidal_velocity(shape, lay.box_len, 1.0, 3.0, 1.0, rng)
    A = [ics.gaussian_filtered_noise(shape, lay.box_len, 0.08, rng) * 0.05 for _ in range(3)]
    bx, by, bz = ics.curl_faces(*A, lay.dx)
    rho = np.exp(0.5 * ics.gaussian_filtered_noise(shape, lay.box_len, 0.1, rng))
    p = 0.6 + 0.1 * rng.random(shape)
    f = ics.Fields(rho=rho, v=v, p=p, bx=bx + 0.7, by=by - 0.3, bz=bz + 0.1, gamma=5.0 / 3.0)
    return f


def test_sums_and_maxima_match_numpy_on_unequal_patch_sizes():
    """Patches of 12 x 10 x 6 (all three sizes differ), 2 x 3 x 4 of them."""
    lay = ics.cartesian((2, 3, 4), (12, 10, 6), dx=1.0 / 24)
    f = _random_state(lay, 3)
    state = ics.to_patches(lay, f)
    got, mdiv, mb = oracle_diag(lay, state)
    tot, scale, mdiv_e, mb_e = expected(lay, state)
    for q in range(8):
        assert abs(got[q] - tot[q]) <= 1e-15 * scale[q], (q, got[q], tot[q])
    assert mdiv == mdiv_e
    assert mb == mb_e
    # a periodic state cut from one global field repeats each upper boundary
    # face as the next patch's low face: the maximum over all stored faces
    assert mb == max(float(np.max(np.abs(a))) for a in state[1:])


def test_planted_face_jumps_are_seen_on_every_face_orientation():
    """On a uniform, divergence-free state, add delta to one face: max |div b|
    becomes exactly |delta| (the face enters two cells' divergences with
    opposite signs, or one cell's when it is a patch's upper boundary face)
    and max |b| moves only when the face is a low face of some cell."""
    lay = ics.cartesian(2, (6, 5, 4), dx=0.1)
    W0 = [1.0, 0.1, -0.2, 0.3, 0.6, 0.5, -0.25, 0.125]
    base = ics.to_patches(lay, ics.config_uniform(lay, W0, 5.0 / 3.0))
    _, mdiv0, mb0 = oracle_diag(lay, base)
    assert mdiv0 == 0.0 and mb0 == 0.5
    delta = 0.75
    ip = 3
    nx, ny, nz = (int(v) for v in lay.n[ip])
    shapes = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
    upper = [(2, 2, nx), (2, ny, 2), (nz, 2, 2)]
    for comp in (1, 2, 3):
        shape = shapes[comp - 1]
        off = ip * int(np.prod(shape))           # every patch has the same size
        for idx in ((2, 2, 2), upper[comp - 1]):
            state = [a.copy() for a in base]
            flat = off + int(np.ravel_multi_index(idx, shape))
            state[comp][flat] += delta
            _, mdiv, mb = oracle_diag(lay, state)
            assert mdiv == delta, (comp, idx, mdiv)
            if idx == (2, 2, 2):
                assert mb == max(mb0, abs(float(state[comp][flat]))), (comp, idx, mb)
            else:
                assert mb == mb0, (comp, idx, mb)   # an upper boundary face is no cell's low face


def test_uniform_state_integrates_to_value_times_volume():
    lay = ics.cartesian(2, 8, dx=1.0 / 16)
    W0 = [1.25, 0.5, -0.25, 0.75, 0.6, 0.5, 0.25, -0.125]
    g = 5.0 / 3.0
    f = ics.config_uniform(lay, W0, g)
    got, mdiv, mb = oracle_diag(lay, ics.to_patches(lay, f), g)
    rho, vx, vy, vz, p, bx, by, bz = W0
    E = p / (g - 1) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    want = [rho, rho * vx, rho * vy, rho * vz, E, bx, by, bz]    # box volume 1
    for q in range(8):
        assert got[q] == pytest.approx(want[q], rel=1e-14, abs=1e-15), q
    assert mdiv == 0.0 and mb == 0.5


def test_two_levels_count_level_one_cells_with_an_eighth_of_the_volume():
    """Level 0: 4^3 patches of 8^3 on the unit box; level 1 over the central
    8^3 level-0 cells (2^3 patches of 8^3 level-1 cells).  A uniform state
    integrates to its value times (1 + (8/32)^3): the level-0 cells under the
    refined region still count, as the diagnostics state."""
    coarse = ics.cartesian(4, 8)
    lay = ics.two_level(coarse, 12, 8, fine_patch=8)
    assert int((lay.levels == 1).sum()) == 8
    g = 5.0 / 3.0
    W0 = [2.0, 0.5, 0.25, -0.5, 0.6, 0.5, -0.25, 0.75]
    rho, vx, vy, vz, p, bx, by, bz = W0
    E = p / (g - 1) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    per = []
    for (nx, ny, nz) in lay.n.astype(int):
        c = nx * ny * nz
        per.append((np.concatenate([np.full(c, v) for v in (rho, rho * vx, rho * vy, rho * vz, E)]),
                    np.full((nx + 1) * ny * nz, bx), np.full(nx * (ny + 1) * nz, by),
                    np.full(nx * ny * (nz + 1), bz)))
    state = [np.concatenate([p_[k] for p_ in per]) for k in range(4)]
    got, mdiv, mb = oracle_diag(lay, state, g)
    vol = 1.0 + (8.0 / 32.0) ** 3
    want = [rho, rho * vx, rho * vy, rho * vz, E, bx, by, bz]
    for q in range(8):
        assert got[q] == pytest.approx(want[q] * vol, rel=1e-14), q
    tot, scale, mdiv_e, mb_e = expected(lay, state)
    for q in range(8):
        assert abs(got[q] - tot[q]) <= 1e-15 * scale[q], q
    assert mdiv == 0.0 and mb == 0.75


def test_two_level_random_state_matches_numpy():
    coarse = ics.cartesian(4, 8)
    lay = ics.two_level(coarse, 12, 8, fine_patch=8)
    rng = np.random.default_rng(8)
    parts = []
    for nx, ny, nz in lay.n.astype(int):
        c = nx * ny * nz
        u = np.concatenate([1.0 + 0.5 * rng.random(c), 0.3 * rng.standard_normal(3 * c), 10.0 + rng.random(c)])
        parts.append((u, 0.5 * rng.standard_normal((nx + 1) * ny * nz), 0.5 * rng.standard_normal(nx * (ny + 1) * nz),
                      0.5 * rng.standard_normal(nx * ny * (nz + 1))))
    state = [np.concatenate([p_[k] for p_ in parts]) for k in range(4)]
    got, mdiv, mb = oracle_diag(lay, state)
    tot, scale, mdiv_e, mb_e = expected(lay, state)
    for q in range(8):
        assert abs(got[q] - tot[q]) <= 1e-15 * scale[q], q
    assert mdiv == mdiv_e and mb == mb_e
