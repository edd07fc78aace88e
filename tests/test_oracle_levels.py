"""Pins of the oracle's two-level guard fill (prolongation and restriction,
DISPATCH I, Sec. 3 A) and of stepping across a resolution jump.

Each check rests on something other than the oracle: data linear in space is
reproduced exactly by any conservative linear interpolation and by averaging
(so every padded box must equal the same linear function sampled at its own
level's cell centres); 8 children of a level-0 cell average to it; a limited
slope vanishes at an extremum; divergence-free faces stay divergence-free
when prolonged piecewise-constantly or restricted by face averaging; a
dyadic uniform state stays exactly uniform; the Courant step halves with the
cell size; and a smooth wave crossing a refined region keeps the accuracy of
the coarse grid.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_1705_10774_gb300 import ics

G53 = 5.0 / 3.0


def make(lay, state, gamma=G53, **kw):
    o = Oracle(lay.n, lay.lo, level=lay.levels, gamma=gamma, cfl=kw.pop("cfl", 0.4),
               base_cells=lay.base_cells, box_len=lay.box_len, **kw)
    o.set_state(*state)
    return o


def layout(coarse_patches=4, n=8, fine_lo=12, fine_cells=8, fine_patch=8):
    """32^3 level 0 (4^3 patches of 8^3) with level 1 over level-0 cells
    [12, 20)^3 (2^3 patches of 8^3 at dx/2): the refined box sits in the middle,
    far from the periodic wrap."""
    return ics.two_level(ics.cartesian(coarse_patches, n), fine_lo, fine_cells, fine_patch=fine_patch)


# linear fields (position in box units)
RHO = lambda x, y, z: 2.0 + 0.3 * x + 0.2 * y + 0.1 * z
VEL = lambda x, y, z: (0.1 + 0 * x, -0.2 + 0 * x, 0.3 + 0 * x)
# face fields varying along their own normal only (divergence-free: 0.2 - 0.2 + 0)
FACES = (lambda x, y, z: 1.0 + 0.2 * x, lambda x, y, z: 0.5 - 0.2 * y, lambda x, y, z: -0.3 + 0 * z)
# pressure chosen so that the total energy is linear too (the magnetic energy
# of the linear field is quadratic)
ELIN = lambda x, y, z: 3.0 + 0.1 * x - 0.2 * y + 0.3 * z
PRE = lambda x, y, z: (G53 - 1) * (ELIN(x, y, z) - 0.5 * RHO(x, y, z) * 0.14
                                  - 0.5 * ((1.0 + 0.2 * x) ** 2 + (0.5 - 0.2 * y) ** 2 + 0.09))


def expected_padded(lay, ip, g=3):
    """The linear fields sampled on patch ip's padded box at its level."""
    n, lo, lev = lay.n[ip], lay.lo[ip], lay.levels[ip]
    sub = ics.Layout(n=(n + 2 * g)[None].astype(np.int32), lo=(lo - g)[None], base_cells=lay.base_cells,
                     box_len=lay.box_len, level=np.array([lev], np.int32))
    U, bx, by, bz = ics.patches_from_functions(sub, RHO, VEL, PRE, G53, faces=FACES)
    N = n + 2 * g
    return (U.reshape(5, N[2], N[1], N[0]), bx.reshape(N[2], N[1], N[0] + 1),
            by.reshape(N[2], N[1] + 1, N[0]), bz.reshape(N[2] + 1, N[1], N[0]))


def test_neighbours_are_symmetric_and_cross_levels():
    lay = layout()
    o = make(lay, ics.patches_from_functions(lay, RHO, VEL, PRE, G53, faces=FACES))
    nb = [set(o.nbors(i).tolist()) for i in range(lay.npatch)]
    lev = lay.levels
    for i in range(lay.npatch):
        for j in nb[i]:
            assert i in nb[j]
    fine = np.flatnonzero(lev == 1)
    coarse = np.flatnonzero(lev == 0)
    for i in fine:   # every level-1 patch reads level 0 around the refined box
        assert any(lev[j] == 0 for j in nb[i])
    # the level-0 patches under and around the refined box [12, 20)^3 see level 1;
    # those far away (e.g. the one at the origin corner's opposite) do not
    far = [i for i in coarse if all(lay.lo[i] == (24, 24, 24))]
    assert far and not any(lev[j] == 1 for j in nb[far[0]])
    near = [i for i in coarse if all(lay.lo[i] == (8, 8, 8))]
    assert near and sum(lev[j] == 1 for j in nb[near[0]]) == len(fine)


def test_linear_data_fills_every_padded_box_exactly():
    """Prolonged level-1 guards and restricted level-0 guards of linear data
    are the linear function at that level's cell and face centres (limited
    slopes of linear data are the exact differences; face fields varying
    along their normal are reproduced by the face rules)."""
    lay = layout()
    o = make(lay, ics.patches_from_functions(lay, RHO, VEL, PRE, G53, faces=FACES))
    lev = lay.levels
    checked = {0: 0, 1: 0}
    for ip in range(lay.npatch):
        L = np.array(lay.base_cells) * 2 ** int(lev[ip])
        if np.any(lay.lo[ip] - 3 < 0) or np.any(lay.lo[ip] + lay.n[ip] + 3 > L):
            continue                    # padded box wraps: linear data are not periodic
        got = o.fill_padded(ip)
        want = expected_padded(lay, ip)
        for a, b in zip(got, want):
            assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b)), (ip, lev[ip])
        checked[int(lev[ip])] += 1
    assert checked[0] == 8 and checked[1] == 8


def test_prolonged_children_average_to_parent_and_flatten_at_extrema():
    """Random level-0 data: the 8 level-1 children of a level-0 cell next to
    the refined box average to the parent (the quarter slopes cancel in
    pairs); at a local extremum of the parent every child equals it."""
    lay = layout()
    rng = np.random.default_rng(3)
    state = list(ics.patches_from_functions(lay, RHO, VEL, PRE, G53, faces=FACES))
    # randomise level-0 densities (keep them positive)
    off = 0
    for ip in range(lay.npatch):
        nc = int(np.prod(lay.n[ip]))
        if lay.levels[ip] == 0:
            state[0][off:off + nc] = 1.0 + rng.random(nc)
        off += 5 * nc
    coarse = {tuple(lay.lo[i]): i for i in range(lay.npatch) if lay.levels[i] == 0}
    U0 = state[0]
    # level-0 cell (11, 13, 14): owner patch lo (8, 8, 8); make it a local maximum
    ipc = coarse[(8, 8, 8)]
    base = 5 * sum(int(np.prod(lay.n[i])) for i in range(ipc))

    def cidx(x, y, z):
        return base + ((z - 8) * 8 + (y - 8)) * 8 + (x - 8)

    U0[cidx(11, 13, 14)] = 5.0
    o = make(lay, state)
    # level-1 patch at fine lo (24, 24, 24): padded box starts at fine cell 21
    ipf = [i for i in range(lay.npatch) if lay.levels[i] == 1 and tuple(lay.lo[i]) == (24, 24, 24)][0]
    Up = o.fill_padded(ipf)[0][0]   # density, (Nz, Ny, Nx), index = fine cell - 21

    def children(X, Y, Z):
        return np.array([Up[2 * Z + c - 21, 2 * Y + b - 21, 2 * X + a - 21]
                         for c in (0, 1) for b in (0, 1) for a in (0, 1)])

    spread = 0.0
    for (X, Y, Z) in [(11, 12, 12), (11, 13, 15), (11, 15, 13), (11, 14, 12)]:
        ch = children(X, Y, Z)
        assert abs(ch.mean() - U0[cidx(X, Y, Z)]) <= 1e-15 * 8
        spread = max(spread, np.ptp(ch))
    assert spread > 0.01               # slopes present
    ch = children(11, 13, 14)
    assert np.all(ch == 5.0)


def _potential(seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 3, size=(3, 3, 3))
    ph = rng.random((3, 3)) * 2 * np.pi

    def comp(c):
        return lambda x, y, z: sum(0.05 * np.sin(2 * np.pi * (k[c, m, 0] * x + k[c, m, 1] * y + k[c, m, 2] * z)
                                                 + ph[c, m]) for m in range(3))
    return comp(0), comp(1), comp(2)


def test_guard_faces_stay_divergence_free_across_levels():
    """Faces from a vector potential (zero divergence per cell on each
    level): padded level-1 cells whose six faces all come from level 0, and
    padded level-0 cells whose six faces all come from level 1, have zero
    divergence."""
    lay = layout()
    A = _potential(11)
    o = make(lay, ics.patches_from_functions(lay, RHO, VEL, PRE, G53, potential=A))
    g = 3
    E = np.eye(3, dtype=np.int64)
    counts = {0: 0, 1: 0}
    for ip in range(lay.npatch):
        lev = int(lay.levels[ip])
        lo, n = lay.lo[ip], lay.n[ip]
        r1 = (24, 40) if lev == 1 else (12, 20)       # the refined box on this level
        in_r1 = lambda c: all(r1[0] <= c[d] < r1[1] for d in range(3))
        interior = lambda c: all(lo[d] <= c[d] < lo[d] + n[d] for d in range(3))
        _, bx, by, bz = o.fill_padded(ip)
        bmax = max(np.abs(bx).max(), np.abs(by).max(), np.abs(bz).max())
        N = n + 2 * g
        for k in range(N[2]):
            for j in range(N[1]):
                for i in range(N[0]):
                    c = lo - g + np.array([i, j, k])
                    if interior(c) or any(interior(c + s * E[d]) for d in range(3) for s in (-1, 1)):
                        continue
                    ups = [c] + [c + E[d] for d in range(3)]
                    cross = all(not in_r1(u) for u in ups) if lev == 1 else all(in_r1(u) for u in ups)
                    if not cross:
                        continue
                    div = (bx[k, j, i + 1] - bx[k, j, i]) + (by[k, j + 1, i] - by[k, j, i]) \
                        + (bz[k + 1, j, i] - bz[k, j, i])
                    assert abs(div) <= 1e-13 * bmax, (ip, c)
                    counts[lev] += 1
    assert counts[0] > 0 and counts[1] > 0


def test_dyadic_uniform_state_stays_exactly_uniform_on_two_levels():
    """Slopes of uniform data vanish and sums of equal dyadic values are
    exact, so prolongation and restriction return the state itself and every
    patch of both levels stays bit-for-bit uniform under local steps; level-1
    steps are exactly half the level-0 steps (same signal speed, half the
    cell size), so level-1 patches update twice as often."""
    lay = layout()
    state = ics.patches_from_functions(
        lay, lambda x, y, z: 1.0 + 0 * x, lambda x, y, z: (0.5 + 0 * x, 0.25 + 0 * x, 0.125 + 0 * x),
        lambda x, y, z: 0.5 + 0 * x, G53,
        faces=(lambda x, y, z: 0.5 + 0 * x, lambda x, y, z: 0.25 + 0 * x, lambda x, y, z: 0 * x))
    o = make(lay, state, time_mode=1)
    o.advance(t_end=2.0 ** -6)          # a multiple of both levels' steps
    for a, b in zip(o.get_state(), state):
        assert np.array_equal(a, b)
    p, t, dt = o.schedule()
    lev = lay.levels[p]
    assert set(np.unique(dt[lev == 1])) == {dt[lev == 0][0] / 2}
    assert len(np.unique(dt[lev == 0])) == 1
    cnt = np.bincount(p, minlength=lay.npatch)
    assert np.all(cnt[lay.levels == 1] == 2 * cnt[lay.levels == 0][0])


def _sound_wave(lay, amp=1e-4, t=0.0):
    """A sound wave along x (rho = 1, p = 0.6, gamma = 5/3: c_s = 1), B = 0."""
    k = 2 * np.pi
    rho = lambda x, y, z: 1.0 + amp * np.sin(k * (x - t))
    vel = lambda x, y, z: (amp * np.sin(k * (x - t)), 0 * x, 0 * x)
    pre = lambda x, y, z: 0.6 + 0.6 * G53 * amp * np.sin(k * (x - t))
    zero = lambda x, y, z: 0 * x
    return ics.patches_from_functions(lay, rho, vel, pre, G53, faces=(zero, zero, zero))


def _density_error(lay, U, t, amp):
    """Volume-weighted L1 error of the density against the travelling wave,
    on level-0 cells outside the refined region and on level-1 cells."""
    err = {0: 0.0, 1: 0.0}
    vol = {0: 0.0, 1: 0.0}
    off = 0
    for ip in range(lay.npatch):
        n, lo, lev = lay.n[ip], lay.lo[ip], int(lay.levels[ip])
        nc = int(np.prod(n))
        h = lay.dx / 2 ** lev
        x = (lo[0] + np.arange(n[0]) + 0.5) * h
        r = U[off:off + nc].reshape(n[2], n[1], n[0])
        ex = 1.0 + amp * np.sin(2 * np.pi * (x - t))
        e = np.abs(r - ex[None, None, :])
        if lev == 0 and lay.levels.max() == 1:
            cx = lo[0] + np.arange(n[0])
            cy = lo[1] + np.arange(n[1])
            cz = lo[2] + np.arange(n[2])
            inside = ((cz[:, None, None] >= 4) & (cz[:, None, None] < 12) & (cy[None, :, None] >= 4)
                      & (cy[None, :, None] < 12) & (cx[None, None, :] >= 4) & (cx[None, None, :] < 12))
            e = e[~inside]
        err[lev] += e.sum() * h ** 3
        vol[lev] += e.size * h ** 3
        off += 5 * nc
    return {k: err[k] / vol[k] for k in err if vol[k] > 0}


def test_sound_wave_crosses_the_refined_box_at_coarse_accuracy():
    """A sound wave on a 16^3 level 0 with level 1 over its central 8^3
    cells: after a quarter period, the error on level 0 stays within 1.5x that
    of the same run without level 1, and the level-1 cells are no worse than
    level 0 (a wrong slope sign or offset in the prolongation, or a wrong
    child in the restriction, shows up as an O(amplitude) jump)."""
    amp, t_end = 1e-4, 0.25
    coarse = ics.cartesian(2, 8)
    two = ics.two_level(coarse, 4, 8, fine_patch=8)
    res = {}
    for name, lay in (("coarse", coarse), ("two", two)):
        o = make(lay, _sound_wave(lay, amp), time_mode=1)
        o.advance(t_end=t_end)
        res[name] = _density_error(lay, o.get_state()[0], t_end, amp)
    e0 = res["coarse"][0]
    assert res["two"][0] <= 1.5 * e0, (res, e0)
    assert res["two"][1] <= 1.0 * e0, (res, e0)


def test_two_level_sweeps_equal_time_sorted_queue():
    """With cross-level neighbours in Eq. (1), the sweep dispatcher and the
    time-sorted ready queue still give bit-identical states and the same
    per-patch schedule (grace 0: ready neighbours share their time, and every
    read touches a neighbour's two newest slices)."""
    lay = layout()
    A = _potential(5)
    rng = np.random.default_rng(2)
    kk = rng.integers(1, 3, size=(3, 3))
    rho = lambda x, y, z: 1.0 + 0.3 * np.sin(2 * np.pi * (kk[0, 0] * x + kk[0, 1] * y + kk[0, 2] * z))
    vel = lambda x, y, z: tuple(0.4 * np.sin(2 * np.pi * (kk[i, 0] * x + kk[i, 1] * y + kk[i, 2] * z) + i)
                                for i in range(3))
    state = ics.patches_from_functions(lay, rho, vel, lambda x, y, z: 0.6 + 0 * x, G53, potential=A)
    runs = []
    for disp in (1, 0):
        o = make(lay, state, time_mode=1, dispatcher=disp)
        o.advance(t_end=0.004)
        runs.append((o.get_state(), sorted(zip(*(x.tolist() for x in o.schedule())))))
    (sa, ka), (sb, kb) = runs
    assert ka == kb
    assert len(set(d for _, _, d in ka)) >= 2
    for a, b in zip(sa, sb):
        assert np.array_equal(a, b)
