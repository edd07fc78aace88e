"""Seeded synthetic inputs: patch layouts and initial states.

This module only *defines inputs*.  It holds none of the update scheme's
arithmetic and is shared by the CUDA path's tests and by the oracle's tests.
Every generator is seeded and returns interior-only patch arrays in the layout
the library uses (x fastest):

    U  : concatenation over patches of [5][nz][ny][nx]  (rho, m_x, m_y, m_z, E)
    bx : concatenation of [nz][ny][nx+1]   (x-faces, both boundary faces)
    by : concatenation of [nz][ny+1][nx]
    bz : concatenation of [nz+1][ny][nx]

Face fields come from a vector potential on cell edges, so their discrete
divergence is zero to round-off.  Units are Heaviside-Lorentz (E = -v x B,
J = curl B), as in DISPATCH I, Sec. 4.3, so E = p/(gamma-1) + rho v^2/2 + B^2/2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Layout:
    """Uniform Cartesian decomposition of a periodic box (DISPATCH I,
    Sec. 2.3, the 'cartesian' component)."""
    n: np.ndarray          # (npatch, 3) int32 cells per axis
    lo: np.ndarray         # (npatch, 3) int64 first interior cell (in its level's index space)
    base_cells: tuple      # level-0 cells per axis (x, y, z)
    box_len: tuple         # box length per axis
    level: np.ndarray = None   # (npatch,) int32 refinement level (0, or 1 at dx/2); None: all 0

    @property
    def npatch(self):
        return self.n.shape[0]

    @property
    def levels(self):
        return np.zeros(self.npatch, np.int32) if self.level is None else np.asarray(self.level, np.int32)

    @property
    def dx(self):
        return self.box_len[0] / self.base_cells[0]


def cartesian(patches_per_axis, cells_per_patch, dx=None):
    """Patches ordered x fastest; cells_per_patch may be an int or a 3-tuple."""
    pp = np.broadcast_to(np.asarray(patches_per_axis, dtype=np.int64), (3,))
    cp = np.broadcast_to(np.asarray(cells_per_patch, dtype=np.int64), (3,))
    base = tuple(int(a * b) for a, b in zip(pp, cp))
    if dx is None:
        dx = 1.0 / base[0]
    box = tuple(float(b * dx) for b in base)
    los = []
    for kz in range(pp[2]):
        for ky in range(pp[1]):
            for kx in range(pp[0]):
                los.append((kx * cp[0], ky * cp[1], kz * cp[2]))
    lo = np.array(los, dtype=np.int64)
    n = np.tile(cp.astype(np.int32), (lo.shape[0], 1))
    return Layout(n=n, lo=lo, base_cells=base, box_len=box)


def mixed_blocks(n_blocks, block=96, sizes=(16, 24, 32), probs=(0.105, 0.266, 0.629), remainder=0,
                 rem_size=32, seed=1, dx=None):
    """Mixed patch sizes on one level: the box is cut into super-blocks of
    `block` cells per axis, each tiled by cubes of one seeded size (volume
    probabilities `probs`; with 16/24/32 and the default probabilities that is
    about 40/30/30 % by patch count); an optional remainder slab of
    `remainder` cells on the high side of every axis is tiled by rem_size
    cubes.  Patches are ordered by super-block, then x fastest inside it."""
    rng = np.random.default_rng(seed)
    L = n_blocks * block + remainder
    if dx is None:
        dx = 1.0 / L
    # the axis segments: super-blocks then the remainder slab
    segs = [(b * block, block) for b in range(n_blocks)]
    if remainder:
        segs.append((n_blocks * block, remainder))
    los, ns = [], []
    for sz_, (z0, zl) in enumerate(segs):
        for (y0, yl) in segs:
            for (x0, xl) in segs:
                if xl == block and yl == block and zl == block:
                    s_ = int(rng.choice(sizes, p=np.asarray(probs) / np.sum(probs)))
                else:
                    s_ = rem_size
                s3 = [s_ if l == block else rem_size for l in (xl, yl, zl)]
                for kz in range(zl // s3[2]):
                    for ky in range(yl // s3[1]):
                        for kx in range(xl // s3[0]):
                            los.append((x0 + kx * s3[0], y0 + ky * s3[1], z0 + kz * s3[2]))
                            ns.append(s3)
    lo = np.array(los, dtype=np.int64)
    n = np.array(ns, dtype=np.int32)
    return Layout(n=n, lo=lo, base_cells=(L, L, L), box_len=(L * dx,) * 3)


def two_level(coarse: Layout, fine_lo, fine_cells, fine_patch=None, fine_n=None, fine_los=None):
    """Two refinement levels (DISPATCH I, Sec. 3 A: patches of differing
    resolution): the level-0 patches of `coarse` and level-1 patches (cell
    size dx/2) tiling the box [fine_lo, fine_lo + fine_cells) given in
    level-0 cells (so every level-1 patch covers whole level-0 cells).  The
    level-1 tiling is either cubes of `fine_patch` cells or explicit
    (fine_n, fine_los) in level-1 cells relative to the box's corner.
    Level-0 patches come first, then level-1 patches (x fastest)."""
    flo = np.broadcast_to(np.asarray(fine_lo, np.int64), (3,))
    fc = np.broadcast_to(np.asarray(fine_cells, np.int64), (3,))
    if fine_n is None:
        m = int(fine_patch)
        assert m % 2 == 0 and all((2 * c) % m == 0 for c in fc)
        los = []
        for kz in range(2 * fc[2] // m):
            for ky in range(2 * fc[1] // m):
                for kx in range(2 * fc[0] // m):
                    los.append((kx * m, ky * m, kz * m))
        fine_los = np.array(los, np.int64)
        fine_n = np.full((len(los), 3), m, np.int32)
    fine_los = np.asarray(fine_los, np.int64).reshape(-1, 3) + 2 * flo
    fine_n = np.asarray(fine_n, np.int32).reshape(-1, 3)
    n = np.concatenate([coarse.n, fine_n]).astype(np.int32)
    lo = np.concatenate([coarse.lo, fine_los]).astype(np.int64)
    level = np.concatenate([coarse.levels, np.ones(len(fine_n), np.int32)])
    return Layout(n=n, lo=lo, base_cells=coarse.base_cells, box_len=coarse.box_len, level=level)


def patches_from_functions(layout: Layout, rho, vel, p, gamma, faces=None, potential=None, dtype=np.float64):
    """Interior-only patch arrays from functions of position, each patch
    sampled on its own level's grid (cell size dx / 2**level): rho(x, y, z),
    vel(x, y, z) -> (vx, vy, vz), p(x, y, z) at cell centres; face fields
    either from `faces` = (bx, by, bz) functions at face centres, or from an
    edge vector potential `potential` = (Ax, Ay, Az) by the discrete curl
    (zero divergence per cell to round-off)."""
    dx0 = layout.dx
    Us, bxs, bys, bzs = [], [], [], []
    for (nx, ny, nz), lo, lev in zip(layout.n, layout.lo, layout.levels):
        h = dx0 / 2 ** int(lev)
        ci = [(lo[d] + np.arange(m) + 0.5) * h for d, m in enumerate((nx, ny, nz))]
        fi = [(lo[d] + np.arange(m + 1)) * h for d, m in enumerate((nx, ny, nz))]
        # coordinates as broadcastable (sparse) grids: functions act elementwise
        Z, Y, X = np.meshgrid(ci[2], ci[1], ci[0], indexing="ij", sparse=True)
        shp = (nz, ny, nx)
        r = np.broadcast_to(rho(X, Y, Z), shp)
        v = [np.broadcast_to(c, shp) for c in vel(X, Y, Z)]
        pr = np.broadcast_to(p(X, Y, Z), shp)
        g = lambda a, b, c: np.meshgrid(c, b, a, indexing="ij", sparse=True)[::-1]
        if faces is not None:
            bx = np.broadcast_to(faces[0](*g(fi[0], ci[1], ci[2])), (nz, ny, nx + 1))
            by = np.broadcast_to(faces[1](*g(ci[0], fi[1], ci[2])), (nz, ny + 1, nx))
            bz = np.broadcast_to(faces[2](*g(ci[0], ci[1], fi[2])), (nz + 1, ny, nx))
        else:
            Ax, Ay, Az = potential
            # x-faces: (Az(y+) - Az(y-)) - (Ay(z+) - Ay(z-)), over h
            bx = ((Az(*g(fi[0], fi[1][1:], ci[2])) - Az(*g(fi[0], fi[1][:-1], ci[2])))
                  - (Ay(*g(fi[0], ci[1], fi[2][1:])) - Ay(*g(fi[0], ci[1], fi[2][:-1])))) / h
            by = ((Ax(*g(ci[0], fi[1], fi[2][1:])) - Ax(*g(ci[0], fi[1], fi[2][:-1])))
                  - (Az(*g(fi[0][1:], fi[1], ci[2])) - Az(*g(fi[0][:-1], fi[1], ci[2])))) / h
            bz = ((Ay(*g(fi[0][1:], ci[1], fi[2])) - Ay(*g(fi[0][:-1], ci[1], fi[2])))
                  - (Ax(*g(ci[0], fi[1][1:], fi[2])) - Ax(*g(ci[0], fi[1][:-1], fi[2])))) / h
            bx = np.broadcast_to(bx, (nz, ny, nx + 1))
            by = np.broadcast_to(by, (nz, ny + 1, nx))
            bz = np.broadcast_to(bz, (nz + 1, ny, nx))
        Bc = (0.5 * (bx[:, :, :-1] + bx[:, :, 1:]), 0.5 * (by[:, :-1] + by[:, 1:]), 0.5 * (bz[:-1] + bz[1:]))
        v2 = v[0] ** 2 + v[1] ** 2 + v[2] ** 2
        E = pr / (gamma - 1.0) + 0.5 * r * v2 + 0.5 * (Bc[0] ** 2 + Bc[1] ** 2 + Bc[2] ** 2)
        Us.append(np.stack([r, r * v[0], r * v[1], r * v[2], E]).ravel())
        bxs.append(np.ascontiguousarray(bx).ravel())
        bys.append(np.ascontiguousarray(by).ravel())
        bzs.append(np.ascontiguousarray(bz).ravel())
    cat = lambda a: np.concatenate(a).astype(dtype)
    return cat(Us), cat(bxs), cat(bys), cat(bzs)


def config_two_level(blocks=5, seed=10774, layout_seeds=(17, 18), dtype=np.float32):
    """The uneven batched solve on two levels: level 0 = (96 blocks + 32)^3
    cells (512^3 for blocks = 5) in 96^3 super-blocks of 16^3 / 24^3 / 32^3
    patches plus 32^3 remainder slabs; level 1 at dx/2 over the central
    quarter-width cube [3/8, 5/8]^3, tiled the same way with its remainder in
    32^3 patches.  Level 0 carries the turbulence input (solenoidal
    E(k) ~ k^-2 on 1 <= |k|/2pi <= 4, rms |v| = 2, rho = 1, p = 0.6, uniform B
    along x at beta = 1); level-1 cells take their level-0 parent's
    velocity.  Returns the layout and the patch arrays (U, bx, by, bz)."""
    coarse = mixed_blocks(blocks, 96, remainder=32, seed=layout_seeds[0])
    X, Y, Z = coarse.base_cells
    fine_lo, fine_cells = 3 * X // 8, X // 4
    fb = 2 * fine_cells // 96
    fine = mixed_blocks(fb, 96, remainder=2 * fine_cells - 96 * fb, seed=layout_seeds[1])
    lay = two_level(coarse, fine_lo, fine_cells, fine_n=fine.n, fine_los=fine.lo)
    rng = np.random.default_rng(seed)
    v = solenoidal_velocity((Z, Y, X), coarse.box_len, 1.0, 4.0, 2.0, rng).astype(np.float32)
    b0 = np.sqrt(1.2)
    f = Fields(rho=np.ones((Z, Y, X)), v=v, p=np.full((Z, Y, X), 0.6), bx=np.full((Z, Y, X), b0),
               by=np.zeros((Z, Y, X)), bz=np.zeros((Z, Y, X)), gamma=5.0 / 3.0)
    s0 = to_patches(coarse, f, dtype=dtype)
    del f
    dx0 = coarse.dx
    par = lambda a: np.clip((a / dx0).astype(np.int64), 0, X - 1)
    vel = lambda x, y, z: (v[0][par(z), par(y), par(x)], v[1][par(z), par(y), par(x)], v[2][par(z), par(y), par(x)])
    fl = Layout(n=fine.n, lo=fine.lo + 2 * fine_lo, base_cells=coarse.base_cells, box_len=coarse.box_len,
                level=np.ones(fine.npatch, np.int32))
    s1 = patches_from_functions(fl, lambda x, y, z: 1.0 + 0 * x, vel, lambda x, y, z: 0.6 + 0 * x, 5.0 / 3.0,
                                faces=(lambda x, y, z: b0 + 0 * x, lambda x, y, z: 0 * x, lambda x, y, z: 0 * x),
                                dtype=dtype)
    return lay, tuple(np.concatenate([a, b]) for a, b in zip(s0, s1))


@dataclass
class Fields:
    """A global periodic state on the level grid (index order z, y, x)."""
    rho: np.ndarray
    v: np.ndarray          # (3, Z, Y, X)
    p: np.ndarray
    bx: np.ndarray         # x-face at i-1/2, periodic: (Z, Y, X)
    by: np.ndarray
    bz: np.ndarray
    gamma: float
    meta: dict = field(default_factory=dict)


def _grid(layout):
    X, Y, Z = layout.base_cells
    dx = layout.dx
    x = (np.arange(X) + 0.5) * dx
    y = (np.arange(Y) + 0.5) * dx
    z = (np.arange(Z) + 0.5) * dx
    return x, y, z, dx


def curl_faces(Ax, Ay, Az, dx):
    """Face fields b = curl A from edge potentials (periodic).

    Ax[k,j,i] sits at (x_i, y_{j-1/2}, z_{k-1/2}), Ay at (x_{i-1/2}, y_j, z_{k-1/2}),
    Az at (x_{i-1/2}, y_{j-1/2}, z_k).  bx[k,j,i] is the face at x_{i-1/2}."""
    bx = (np.roll(Az, -1, axis=1) - Az) / dx - (np.roll(Ay, -1, axis=0) - Ay) / dx
    by = (np.roll(Ax, -1, axis=0) - Ax) / dx - (np.roll(Az, -1, axis=2) - Az) / dx
    bz = (np.roll(Ay, -1, axis=2) - Ay) / dx - (np.roll(Ax, -1, axis=1) - Ax) / dx
    return bx, by, bz


def to_patches(layout: Layout, f: Fields, dtype=np.float64):
    """Cut the global state into interior-only patch arrays (conserved U)."""
    Bxc = 0.5 * (f.bx + np.roll(f.bx, -1, axis=2))
    Byc = 0.5 * (f.by + np.roll(f.by, -1, axis=1))
    Bzc = 0.5 * (f.bz + np.roll(f.bz, -1, axis=0))
    v2 = f.v[0] ** 2 + f.v[1] ** 2 + f.v[2] ** 2
    E = f.p / (f.gamma - 1.0) + 0.5 * f.rho * v2 + 0.5 * (Bxc ** 2 + Byc ** 2 + Bzc ** 2)
    Ug = np.stack([f.rho, f.rho * f.v[0], f.rho * f.v[1], f.rho * f.v[2], E])
    Z, Y, X = f.rho.shape

    def cut(a, starts, lens):
        """a[..., z0:z0+lz, y0:y0+ly, x0:x0+lx] on the periodic grid (views
        unless an axis wraps)."""
        nd = a.ndim
        for ax, (s0, ln) in enumerate(zip(starts, lens)):
            axis = nd - 3 + ax
            N = a.shape[axis]
            if s0 + ln <= N:
                a = a[(slice(None),) * axis + (slice(s0, s0 + ln),)]
            else:
                a = np.take(a, np.arange(s0, s0 + ln) % N, axis=axis)
        return a

    Us, bxs, bys, bzs = [], [], [], []
    for (nx, ny, nz), (x0, y0, z0) in zip(layout.n, layout.lo):
        Us.append(cut(Ug, (z0, y0, x0), (nz, ny, nx)).ravel())
        bxs.append(cut(f.bx, (z0, y0, x0), (nz, ny, nx + 1)).ravel())
        bys.append(cut(f.by, (z0, y0, x0), (nz, ny + 1, nx)).ravel())
        bzs.append(cut(f.bz, (z0, y0, x0), (nz + 1, ny, nx)).ravel())
    cat = lambda a: np.concatenate(a).astype(dtype)
    return cat(Us), cat(bxs), cat(bys), cat(bzs)


def from_patches(layout: Layout, U, bx, by, bz):
    """Reassemble global cell arrays (U on cells, faces at i-1/2) from patch
    arrays; the inverse of to_patches for a full tiling."""
    X, Y, Z = layout.base_cells
    Ug = np.zeros((5, Z, Y, X))
    bxg = np.zeros((Z, Y, X)); byg = np.zeros((Z, Y, X)); bzg = np.zeros((Z, Y, X))
    oU = ox = oy = oz = 0
    for (nx, ny, nz), (x0, y0, z0) in zip(layout.n, layout.lo):
        nc = nx * ny * nz
        u = np.asarray(U[oU:oU + 5 * nc]).reshape(5, nz, ny, nx)
        fx = np.asarray(bx[ox:ox + (nx + 1) * ny * nz]).reshape(nz, ny, nx + 1)
        fy = np.asarray(by[oy:oy + nx * (ny + 1) * nz]).reshape(nz, ny + 1, nx)
        fz = np.asarray(bz[oz:oz + nx * ny * (nz + 1)]).reshape(nz + 1, ny, nx)
        sl = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
        Ug[(slice(None),) + sl] = u
        bxg[sl] = fx[:, :, :nx]
        byg[sl] = fy[:, :ny, :]
        bzg[sl] = fz[:nz]
        oU += 5 * nc; ox += (nx + 1) * ny * nz; oy += nx * (ny + 1) * nz; oz += nx * ny * (nz + 1)
    return Ug, bxg, byg, bzg


# ---------------------------------------------------------------- linear MHD

def primitive_jacobian(W0, khat, gamma):
    """A(k) = sum_d khat_d A_d of ideal MHD in primitive variables
    (rho, v, p, B) about a uniform state, with div B = 0 assumed.  Its
    eigenvectors define the linear wave families used as inputs."""
    rho, v, p, B = W0[0], W0[1:4], W0[4], W0[5:8]
    A = np.zeros((8, 8))
    for d in range(3):
        Ad = np.zeros((8, 8))
        Ad[0, 0] = v[d]; Ad[0, 1 + d] = rho
        for c in range(3):
            Ad[1 + c, 1 + c] += v[d]
            Ad[1 + c, 5 + c] -= B[d] / rho
        Ad[1 + d, 4] += 1.0 / rho
        for e in range(3):
            Ad[1 + d, 5 + e] += B[e] / rho
        Ad[4, 4] = v[d]; Ad[4, 1 + d] = gamma * p
        for c in range(3):
            Ad[5 + c, 1 + c] -= B[d]
            Ad[5 + c, 5 + c] += v[d]
            Ad[5 + c, 1 + d] += B[c]
        A += khat[d] * Ad
    return A


def eigenmode(W0, khat, gamma, kind):
    """Right eigenvector (unit norm, real) and speed of a wave family moving
    along +khat: kind in {'fast', 'alfven', 'slow'}."""
    A = primitive_jacobian(W0, khat, gamma)
    lam, R = np.linalg.eig(A)
    lam = lam.real
    R = R.real
    vn = float(np.dot(W0[1:4], khat))
    pos = [i for i in range(8) if lam[i] - vn > 1e-9]
    pos.sort(key=lambda i: lam[i])
    if len(pos) != 3:
        raise ValueError("degenerate wave families for this direction")
    i = {"slow": pos[0], "alfven": pos[1], "fast": pos[2]}[kind]
    r = R[:, i] / np.linalg.norm(R[:, i])
    if r[np.argmax(np.abs(r))] < 0:
        r = -r
    return r, lam[i]


def linear_modes(layout, modes, W0, gamma, amplitude):
    """Superposition of linear eigenmodes.  modes: list of (kind, n_vec,
    phase) with wavevector k = 2 pi n / box.  The field perturbation is set
    through an edge vector potential so that div b = 0 discretely."""
    x, y, z, dx = _grid(layout)
    X, Y, Z = layout.base_cells
    L = np.array(layout.box_len)
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    xe = np.arange(X) * dx
    ye = np.arange(Y) * dx
    ze = np.arange(Z) * dx
    rho = np.full((Z, Y, X), W0[0]); p = np.full((Z, Y, X), W0[4])
    v = np.zeros((3, Z, Y, X)); v += np.asarray(W0[1:4])[:, None, None, None]
    Ax = np.zeros((Z, Y, X)); Ay = np.zeros((Z, Y, X)); Az = np.zeros((Z, Y, X))
    for kind, nvec, phase in modes:
        k = 2 * np.pi * np.asarray(nvec, float) / L
        kh = k / np.linalg.norm(k)
        r, _ = eigenmode(np.asarray(W0, float), kh, gamma, kind)
        th = k[0] * xx + k[1] * yy + k[2] * zz + phase
        cs = amplitude * np.cos(th)
        rho += r[0] * cs
        for c in range(3):
            v[c] += r[1 + c] * cs
        p += r[4] * cs
        dB = amplitude * r[5:8]
        # curl(a sin(k.x + phase)) = (k x a) cos(...) = dB cos(...) for a = -(k x dB)/k^2
        Avec = -np.cross(k, dB) / np.dot(k, k)
        zg, yg, xg = np.meshgrid(ze, ye, x, indexing="ij")
        Ax += Avec[0] * np.sin(k[0] * xg + k[1] * yg + k[2] * zg + phase)
        zg, yg, xg = np.meshgrid(ze, y, xe, indexing="ij")
        Ay += Avec[1] * np.sin(k[0] * xg + k[1] * yg + k[2] * zg + phase)
        zg, yg, xg = np.meshgrid(z, ye, xe, indexing="ij")
        Az += Avec[2] * np.sin(k[0] * xg + k[1] * yg + k[2] * zg + phase)
    bx, by, bz = curl_faces(Ax, Ay, Az, dx)
    bx = bx + W0[5]; by = by + W0[6]; bz = bz + W0[7]
    return Fields(rho=rho, v=v, p=p, bx=bx, by=by, bz=bz, gamma=gamma)


def config_linear_waves(seed=1705, patches=2, n=16, amplitude=1e-6):
    """Eight patches of 16^3 on the unit periodic cube, rho=1, p=0.6, B=(1,0,0),
    v=0, plus four seeded linear fast/Alfven/slow modes with integer
    wavenumbers 1 <= |n| <= 2 (never parallel to x) and random phases."""
    rng = np.random.default_rng(seed)
    lay = cartesian(patches, n)
    W0 = np.array([1.0, 0, 0, 0, 0.6, 1.0, 0, 0])
    modes = []
    while len(modes) < 4:
        nv = rng.integers(-2, 3, size=3)
        nn = np.linalg.norm(nv)
        if nn < 1 or nn > 2 or (nv[1] == 0 and nv[2] == 0):
            continue
        kind = ["fast", "alfven", "slow"][rng.integers(0, 3)]
        phase = rng.uniform(0, 2 * np.pi)
        try:   # skip directions (e.g. k normal to B) where the families coincide
            eigenmode(W0, nv / nn, 5.0 / 3.0, kind)
        except ValueError:
            continue
        modes.append((kind, nv, phase))
    f = linear_modes(lay, modes, W0, 5.0 / 3.0, amplitude)
    f.meta = dict(modes=modes)
    return lay, f


# ------------------------------------------------------- turbulence inputs

def solenoidal_velocity(shape, box, kmin, kmax, rms, rng):
    """Gaussian random solenoidal velocity with shell spectrum E(k) ~ k^-2 on
    kmin <= |k|/2pi <= kmax (so |v_hat| ~ k^-2), zero mean, scaled to the
    given volume rms of |v|."""
    Z, Y, X = shape
    kz = np.fft.fftfreq(Z, d=box[2] / Z)
    ky = np.fft.fftfreq(Y, d=box[1] / Y)
    kx = np.fft.rfftfreq(X, d=box[0] / X)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    band = (K >= kmin) & (K <= kmax)
    amp = np.zeros_like(K)
    amp[band] = K[band] ** -2.0
    vh = [(rng.standard_normal(K.shape) + 1j * rng.standard_normal(K.shape)) * amp for _ in range(3)]
    Ks = np.where(K > 0, K, 1.0)
    kd = (KX * vh[0] + KY * vh[1] + KZ * vh[2]) / Ks ** 2
    vh = [vh[0] - KX * kd, vh[1] - KY * kd, vh[2] - KZ * kd]
    v = np.stack([np.fft.irfftn(c, s=shape, axes=(0, 1, 2)) for c in vh])
    v -= v.mean(axis=(1, 2, 3), keepdims=True)
    r = np.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    return v * (rms / r)


def config_turbulence(seed=10774, patches=8, n=32, mach=2.0):
    """Decaying-turbulence input: 8^3 patches of 32^3 (256^3 cells), rho=1,
    p=0.6 (sound speed 1), solenoidal Gaussian velocity with E(k) ~ k^-2 on
    1 <= |k|/2pi <= 4 at rms Mach 2, uniform B along x with beta = 1."""
    rng = np.random.default_rng(seed)
    lay = cartesian(patches, n)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    v = solenoidal_velocity(shape, lay.box_len, 1.0, 4.0, mach, rng)
    rho = np.ones(shape)
    p = np.full(shape, 0.6)
    B0 = np.sqrt(2 * 0.6 / 1.0)       # beta = 2p/B^2 = 1
    f = Fields(rho=rho, v=v, p=p, bx=np.full(shape, B0), by=np.zeros(shape), bz=np.zeros(shape),
               gamma=5.0 / 3.0)
    return lay, f


def gaussian_filtered_noise(shape, box, sigma_f, rng):
    Z, Y, X = shape
    w = rng.standard_normal(shape)
    kz = np.fft.fftfreq(Z, d=box[2] / Z) * 2 * np.pi
    ky = np.fft.fftfreq(Y, d=box[1] / Y) * 2 * np.pi
    kx = np.fft.rfftfreq(X, d=box[0] / X) * 2 * np.pi
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    g = np.fft.irfftn(np.fft.rfftn(w) * np.exp(-0.5 * (KX ** 2 + KY ** 2 + KZ ** 2) * sigma_f ** 2), s=shape, axes=(0, 1, 2))
    g -= g.mean()
    return g / g.std()


def config_lts(seed=17051, patches=16, n=16, sigma_ln=1.5, hot_radius=0.1, hot_factor=1000.0,
               mach=1.0, beta=10.0, edge_cells=2.0):
    """Local-time-step stress input: log-normal density (sigma_ln = 1.5,
    Gaussian-filtered noise, filter width 1/16 of the box) in pressure
    equilibrium p = 0.6, a central sphere of radius 0.1 at 1000x temperature
    (density / 1000, the edge smoothed over 2 cells), random solenoidal
    velocity at rms Mach 1 with the local sound speed (volume rms of
    |v|/c_s = 1), uniform B along x at beta = 10."""
    rng = np.random.default_rng(seed)
    lay = cartesian(patches, n)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    x, y, zc, _ = _grid(lay)
    g = gaussian_filtered_noise(shape, lay.box_len, lay.box_len[0] / 16.0, rng)
    rho = np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    zz, yy, xx = np.meshgrid(zc, y, x, indexing="ij")
    c = np.array(lay.box_len) / 2
    r2 = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2
    # temperature contrast hot_factor inside the sphere, its edge smoothed
    # over `edge_cells` cells with a tanh profile (in log density)
    if edge_cells > 0:
        w = 0.5 * (1.0 - np.tanh((np.sqrt(r2) - hot_radius) / (edge_cells * lay.dx)))
        rho = rho * np.exp(-np.log(hot_factor) * w)
    else:
        rho = np.where(r2 < hot_radius ** 2, rho / hot_factor, rho)
    p = np.full(shape, 0.6)
    # rms Mach number taken with the local sound speed: scale the solenoidal
    # field so that the volume rms of |v| / c_s(x) is `mach`
    v = solenoidal_velocity(shape, lay.box_len, 1.0, 4.0, 1.0, rng)
    cs = np.sqrt(5.0 / 3.0 * p / rho)
    v *= mach / np.sqrt(np.mean((v[0] ** 2 + v[1] ** 2 + v[2] ** 2) / cs ** 2))
    B0 = np.sqrt(2 * 0.6 / beta)
    f = Fields(rho=rho, v=v, p=p, bx=np.full(shape, B0), by=np.zeros(shape), bz=np.zeros(shape),
               gamma=5.0 / 3.0)
    return lay, f


def config_orszag_tang(seed=10775, patches=16, n=32, pert=1e-3):
    """3-D Orszag-Tang-type vortex: rho = 25/(36 pi), p = 5/(12 pi),
    v = (-sin 2 pi y, sin 2 pi x, 0), b = curl(A_z z) with
    A_z = B0 (cos 4 pi x / 4 pi + cos 2 pi y / 2 pi), B0 = 1/sqrt(4 pi),
    and a seeded 1e-3 Gaussian v_z per cell."""
    rng = np.random.default_rng(seed)
    lay = cartesian(patches, n)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    x, y, z, dx = _grid(lay)
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    rho = np.full(shape, 25.0 / (36.0 * np.pi))
    p = np.full(shape, 5.0 / (12.0 * np.pi))
    v = np.zeros((3,) + shape)
    v[0] = -np.sin(2 * np.pi * yy)
    v[1] = np.sin(2 * np.pi * xx)
    v[2] = pert * rng.standard_normal(shape)
    B0 = 1.0 / np.sqrt(4 * np.pi)
    xe = np.arange(X) * dx
    ye = np.arange(Y) * dx
    _, YE, XE = np.meshgrid(z, ye, xe, indexing="ij")
    Az = B0 * (np.cos(4 * np.pi * XE) / (4 * np.pi) + np.cos(2 * np.pi * YE) / (2 * np.pi))
    zero = np.zeros(shape)
    bx, by, bz = curl_faces(zero, zero, Az, dx)
    return lay, Fields(rho=rho, v=v, p=p, bx=bx, by=by, bz=bz, gamma=5.0 / 3.0)


def orszag_tang_patches(seed=10775, patches=16, n=32, pert=1e-3):
    """The patch arrays of config_orszag_tang, cut directly into patches
    without the global 3-D fields (which at 512^3 take tens of GB): every
    field but the random v_z is independent of z, so faces, velocities and
    the magnetic energy are built on the (y, x) plane and broadcast, and the
    random v_z is drawn exactly as config_orszag_tang draws it.  The values
    equal to_patches(*config_orszag_tang(...)) bit for bit (same elementwise
    operations).  Returns (layout, (U, bx, by, bz))."""
    rng = np.random.default_rng(seed)
    lay = cartesian(patches, n)
    X, Y, Z = lay.base_cells
    x, y, z, dx = _grid(lay)
    rho = 25.0 / (36.0 * np.pi)
    p = 5.0 / (12.0 * np.pi)
    gamma = 5.0 / 3.0
    vz = pert * rng.standard_normal((Z, Y, X))
    B0 = 1.0 / np.sqrt(4 * np.pi)
    xe = np.arange(X) * dx
    ye = np.arange(Y) * dx
    YE, XE = np.meshgrid(ye, xe, indexing="ij")
    Az = B0 * (np.cos(4 * np.pi * XE) / (4 * np.pi) + np.cos(2 * np.pi * YE) / (2 * np.pi))
    bx2 = (np.roll(Az, -1, axis=0) - Az) / dx - 0.0
    by2 = 0.0 - (np.roll(Az, -1, axis=1) - Az) / dx
    yy, xx = np.meshgrid(y, x, indexing="ij")
    vx2 = -np.sin(2 * np.pi * yy)
    vy2 = np.sin(2 * np.pi * xx)
    Bxc = 0.5 * (bx2 + np.roll(bx2, -1, axis=1))
    Byc = 0.5 * (by2 + np.roll(by2, -1, axis=0))
    Bzc = 0.5 * (np.zeros_like(bx2) + np.zeros_like(bx2))
    me2 = Bxc ** 2 + Byc ** 2 + Bzc ** 2
    P = patches
    npch = P ** 3

    def blocks(a):
        """(Z, Y, X) -> (npatch, n, n, n), patches x fastest."""
        return a.reshape(P, n, P, n, P, n).transpose(0, 2, 4, 1, 3, 5).reshape(npch, n, n, n)

    def blocks2(a):
        """(Y, X) plane -> (npatch, n, n, n) broadcast over z."""
        b = a.reshape(P, n, P, n).transpose(0, 2, 1, 3)            # (py, px, ny, nx)
        return np.broadcast_to(b[None, :, :, None], (P, P, P, n, n, n)).reshape(npch, n, n, n)

    U = np.empty((npch, 5, n, n, n))
    VZ = blocks(vz)
    del vz
    U[:, 0] = rho
    U[:, 1] = blocks2(rho * vx2)
    U[:, 2] = blocks2(rho * vy2)
    U[:, 3] = rho * VZ
    vx = blocks2(vx2)
    vy = blocks2(vy2)
    U[:, 4] = p / (gamma - 1.0) + 0.5 * rho * (vx ** 2 + vy ** 2 + VZ ** 2) + 0.5 * blocks2(me2)
    del VZ, vx, vy
    # faces of each patch (both boundary faces), periodic wrap at the box edge
    cx = (np.arange(P)[:, None] * n + np.arange(n + 1)[None, :]) % X      # (px, n+1)
    rw = (np.arange(P)[:, None] * n + np.arange(n)[None, :])              # (py, n)
    fx = bx2[rw[:, None, :, None], cx[None, :, None, :]]                   # (py, px, n, n+1)
    bx = np.broadcast_to(fx[None, :, :, None], (P, P, P, n, n, n + 1)).reshape(-1)
    ry = (np.arange(P)[:, None] * n + np.arange(n + 1)[None, :]) % Y       # (py, n+1)
    cl = (np.arange(P)[:, None] * n + np.arange(n)[None, :])               # (px, n)
    fy = by2[ry[:, None, :, None], cl[None, :, None, :]]                   # (py, px, n+1, n)
    by = np.broadcast_to(fy[None, :, :, None], (P, P, P, n, n + 1, n)).reshape(-1)
    bz = np.zeros(npch * (n + 1) * n * n)
    return lay, (U.reshape(-1), np.ascontiguousarray(bx), np.ascontiguousarray(by), bz)


def config_uniform(layout, W0, gamma, seed=0, eps=0.0):
    """Uniform state plus an optional seeded cell-wise density perturbation."""
    rng = np.random.default_rng(seed)
    X, Y, Z = layout.base_cells
    shape = (Z, Y, X)
    rho = np.full(shape, W0[0]) * (1.0 + eps * rng.standard_normal(shape))
    v = np.zeros((3,) + shape) + np.asarray(W0[1:4])[:, None, None, None]
    return Fields(rho=rho, v=v, p=np.full(shape, W0[4]), bx=np.full(shape, W0[5]), by=np.full(shape, W0[6]),
                  bz=np.full(shape, W0[7]), gamma=gamma)


def config_sod(axis, n_per_unit, cells_per_patch=64, thin=4):
    """Sod tube along `axis` on a periodic box of length 2 (left state
    (rho, p) = (1, 1) on [0.5, 1.5), right state (0.125, 0.1) elsewhere,
    gamma = 1.4, B = 0): the standard Sod interface sits at 1.5, and the waves
    of the mirrored interface at 0.5 stay clear of [1, 2) until t = 0.2."""
    N = 2 * n_per_unit
    cpp = [thin, thin, thin]
    cpp[axis] = cells_per_patch
    ppa = [1, 1, 1]
    ppa[axis] = N // cells_per_patch
    lay = cartesian(ppa, cpp, dx=1.0 / n_per_unit)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    coords = _grid(lay)[axis]
    s = [1, 1, 1]
    s[2 - axis] = -1
    c = coords.reshape(s)
    left = (c >= 0.5) & (c < 1.5)
    rho = np.broadcast_to(np.where(left, 1.0, 0.125), shape).copy()
    p = np.broadcast_to(np.where(left, 1.0, 0.1), shape).copy()
    z = np.zeros(shape)
    return lay, Fields(rho=rho, v=np.zeros((3,) + shape), p=p, bx=z.copy(), by=z.copy(), bz=z.copy(), gamma=1.4)
