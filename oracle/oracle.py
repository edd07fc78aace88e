"""ctypes wrapper around the C oracle (``dispatch_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is a plain, slow FP64 CPU program of the
same method as the CUDA path, written independently of it.  It is imported by
the tests, by the smoke check and by the CPU-baseline leg of the benchmark,
never by the product path.

The oracle follows DISPATCH I (Nordlund et al. 2018): patches with guard zones
filled by linear (or quadratic) time inter- and extrapolation (Sec. 3 A and
B), readiness by Eq. (1) with grace g, a time-sorted ready queue (Sec. 3 B)
and local Courant steps
(Sec. 5.1); the MHD step is MUSCL-Hancock with HLL fluxes and constrained
transport (Secs. 4.1 and 4.3 name the solver family; the scheme itself is the
textbook one), optionally HLLD fluxes and the non-ideal Ohmic and ambipolar
terms of Sec. 4.3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dispatch_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

D = ctypes.c_double
I32 = ctypes.c_int32
I64 = ctypes.c_int64
P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_create.restype = P
            L.orc_create.argtypes = [ctypes.c_int, P, P, P, D, D, D, D, P, P,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_destroy.argtypes = [P]
            L.orc_set_state.argtypes = [P, P, P, P, P]
            L.orc_set_slot.argtypes = [P, ctypes.c_int, ctypes.c_int, D, P, P, P, P]
            L.orc_set_latest.argtypes = [P, ctypes.c_int, ctypes.c_int, D]
            L.orc_get_state.argtypes = [P, P, P, P, P]
            L.orc_get_times.argtypes = [P, P, P, P]
            L.orc_advance.argtypes = [P, D, I64]
            L.orc_get_schedule.restype = I64
            L.orc_get_schedule.argtypes = [P, P, P, P, I64]
            L.orc_stats.argtypes = [P, P]
            L.orc_diagnostics.argtypes = [P, P]
            L.orc_patch_dt.argtypes = [P, ctypes.c_int, D, P]
            L.orc_update_patch.argtypes = [P, ctypes.c_int, D, P, P, P, P, P]
            L.orc_num_nbors.argtypes = [P, ctypes.c_int, P]
            L.orc_fill_padded.argtypes = [P, ctypes.c_int, P, P, P, P]
            L.orc_set_riemann.argtypes = [P, ctypes.c_int]
            L.orc_set_nonideal.argtypes = [P, D, D, D, D, D]
            L.orc_set_time.argtypes = [P, D, ctypes.c_int]
            L.orc_hlld.argtypes = [P, P, ctypes.c_int, D, P, P]
            L.orc_hlld_fan.argtypes = [P, P, ctypes.c_int, D, P]
            L.orc_last_error.restype = ctypes.c_char_p
            L.orc_last_error.argtypes = [P]
            L.orc_prim.argtypes = [P, P, D, P]
            L.orc_cfast.restype = D
            L.orc_cfast.argtypes = [D, D, D, D, D, D]
            L.orc_mc.restype = D
            L.orc_mc.argtypes = [D, D]
            L.orc_predict.argtypes = [P, P, P, P, D, D, P]
            L.orc_hll.argtypes = [P, P, ctypes.c_int, D, P, P]
            L.orc_emf.restype = D
            L.orc_emf.argtypes = [P, P, P, P, ctypes.c_int, D, D, D, D]
            L.orc_pow2_floor.restype = D
            L.orc_pow2_floor.argtypes = [D]
            L.orc_set_owned.argtypes = [P, P]
            L.orc_get_newest.argtypes = [P, ctypes.c_int, P, P, P, P, P]
            L.orc_push_slice.argtypes = [P, ctypes.c_int, P, P, P, P, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One oracle context: a set of patches on a periodic box, on level 0
    and optionally level 1 (half the cell size).

    ``n`` and ``lo`` are (npatch, 3) integer arrays (cells per axis, first
    interior cell in the patch's level's index space, axis order x, y, z);
    ``level`` is an optional (npatch,) array of 0 / 1.
    """

    def __init__(self, n, lo, *, level=None, gamma, cfl, base_cells, box_len=(1.0, 1.0, 1.0), t0=0.0,
                 dt_max=0.0, nguard=3, nslices=3, time_mode=0, dispatcher=1, riemann=0, eta=0.0,
                 gamma_ad=0.0, rho_i=1.0, c_ohm=0.1, c_ad=0.1, grace=0.0, time_order=1):
        L = lib()
        self.n = np.ascontiguousarray(n, dtype=np.int32).reshape(-1, 3)
        self.lo = np.ascontiguousarray(lo, dtype=np.int64).reshape(-1, 3)
        self.np = self.n.shape[0]
        self.level = (np.zeros(self.np, dtype=np.int32) if level is None
                      else np.ascontiguousarray(level, dtype=np.int32).reshape(-1))
        bl = _f64(box_len)
        bc = np.ascontiguousarray(base_cells, dtype=np.int32)
        h = L.orc_create(self.np, _ptr(self.n), _ptr(self.lo), _ptr(self.level), gamma, cfl, t0, dt_max,
                         _ptr(bl), _ptr(bc), nguard, nslices, time_mode, dispatcher)
        if not h:
            raise ValueError("oracle rejected the layout or parameters")
        self._h = h
        self._check(L.orc_set_riemann(h, riemann))
        # non-ideal MHD (Sec. 4.3): Ohmic resistivity eta, ambipolar drift
        # coefficient gamma_ad with ion density rho_i; 0 turns a term off
        self._check(L.orc_set_nonideal(h, eta, gamma_ad, rho_i, c_ohm, c_ad))
        # grace of Eq. 1 and the order of the time inter- and extrapolation
        self._check(L.orc_set_time(h, grace, time_order))
        self.gamma = gamma
        self.nslices = nslices
        nc = self.n[:, 0].astype(np.int64) * self.n[:, 1] * self.n[:, 2]
        self.ncell = nc
        self.nfx = (self.n[:, 0] + 1).astype(np.int64) * self.n[:, 1] * self.n[:, 2]
        self.nfy = self.n[:, 0].astype(np.int64) * (self.n[:, 1] + 1) * self.n[:, 2]
        self.nfz = self.n[:, 0].astype(np.int64) * self.n[:, 1] * (self.n[:, 2] + 1)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError("oracle error %d: %s" % (rc, lib().orc_last_error(self._h).decode()))

    def set_state(self, U, bx, by, bz):
        U, bx, by, bz = (_f64(a) for a in (U, bx, by, bz))
        assert U.size == 5 * self.ncell.sum() and bx.size == self.nfx.sum()
        assert by.size == self.nfy.sum() and bz.size == self.nfz.sum()
        self._check(lib().orc_set_state(self._h, _ptr(U), _ptr(bx), _ptr(by), _ptr(bz)))

    def set_slot(self, ip, s, t, U, bx, by, bz):
        U, bx, by, bz = (_f64(a) for a in (U, bx, by, bz))
        self._check(lib().orc_set_slot(self._h, ip, s, t, _ptr(U), _ptr(bx), _ptr(by), _ptr(bz)))

    def set_latest(self, ip, s, dt_last=0.0):
        self._check(lib().orc_set_latest(self._h, ip, s, dt_last))

    def get_state(self):
        U = np.empty(5 * self.ncell.sum())
        bx = np.empty(self.nfx.sum())
        by = np.empty(self.nfy.sum())
        bz = np.empty(self.nfz.sum())
        self._check(lib().orc_get_state(self._h, _ptr(U), _ptr(bx), _ptr(by), _ptr(bz)))
        return U, bx, by, bz

    def get_times(self):
        t = np.empty(self.np)
        dt = np.empty(self.np)
        sm = np.empty(self.np)
        lib().orc_get_times(self._h, _ptr(t), _ptr(dt), _ptr(sm))
        return t, dt, sm

    def advance(self, t_end=float("inf"), max_sweeps=0):
        self._check(lib().orc_advance(self._h, t_end, max_sweeps))

    def schedule(self):
        n = lib().orc_get_schedule(self._h, None, None, None, 0)
        p = np.empty(n, np.int64)
        t = np.empty(n)
        dt = np.empty(n)
        lib().orc_get_schedule(self._h, _ptr(p), _ptr(t), _ptr(dt), n)
        return p, t, dt

    def stats(self):
        out = np.zeros(5, np.int64)
        lib().orc_stats(self._h, _ptr(out))
        return dict(patch_updates=int(out[0]), cell_updates=int(out[1]), sweeps=int(out[2]),
                    fallbacks=int(out[3]), floors=int(out[4]))

    def diagnostics(self):
        out = np.zeros(10)
        lib().orc_diagnostics(self._h, _ptr(out))
        return dict(mass=out[0], mom=out[1:4].copy(), energy=out[4], bmean=out[5:8].copy(),
                    max_divb=out[8], max_b=out[9])

    def patch_dt(self, ip, t_end=float("inf")):
        dt = np.zeros(1)
        self._check(lib().orc_patch_dt(self._h, ip, t_end, _ptr(dt)))
        return float(dt[0])

    def update_patch(self, ip, dt):
        nc, fx, fy, fz = self.ncell[ip], self.nfx[ip], self.nfy[ip], self.nfz[ip]
        U = np.empty(5 * nc)
        bx = np.empty(fx)
        by = np.empty(fy)
        bz = np.empty(fz)
        sm = np.zeros(1)
        self._check(lib().orc_update_patch(self._h, ip, dt, _ptr(U), _ptr(bx), _ptr(by), _ptr(bz), _ptr(sm)))
        return U, bx, by, bz, float(sm[0])

    def set_owned(self, owned):
        """Sec. 3 C: owned[i] = 1 for a patch this process updates, 0 for a
        virtual copy of a patch another process owns."""
        o = np.ascontiguousarray(owned, dtype=np.int8)
        assert o.size == self.np
        self._check(lib().orc_set_owned(self._h, _ptr(o)))

    def newest(self, ip):
        """The package of patch ip: (U, bx, by, bz) of its newest slice and
        (time, last step, signal speed)."""
        U = np.empty(5 * self.ncell[ip])
        bx = np.empty(self.nfx[ip])
        by = np.empty(self.nfy[ip])
        bz = np.empty(self.nfz[ip])
        meta = np.empty(3)
        self._check(lib().orc_get_newest(self._h, ip, _ptr(U), _ptr(bx), _ptr(by), _ptr(bz), _ptr(meta)))
        return (U, bx, by, bz), meta

    def push(self, ip, arrays, meta):
        """Store a received package as the newest slice of virtual patch ip."""
        U, bx, by, bz = (_f64(a) for a in arrays)
        meta = _f64(meta)
        self._check(lib().orc_push_slice(self._h, ip, _ptr(U), _ptr(bx), _ptr(by), _ptr(bz), _ptr(meta)))

    def fill_padded(self, ip, nguard=3):
        """The padded box of patch ip at its current time (guard depth
        nguard): U (5, Nz, Ny, Nx), bx (Nz, Ny, Nx+1), by (Nz, Ny+1, Nx),
        bz (Nz+1, Ny, Nx)."""
        nx, ny, nz = (int(a) + 2 * nguard for a in self.n[ip])
        U = np.zeros((5, nz, ny, nx))
        bx = np.zeros((nz, ny, nx + 1))
        by = np.zeros((nz, ny + 1, nx))
        bz = np.zeros((nz + 1, ny, nx))
        self._check(lib().orc_fill_padded(self._h, ip, _ptr(U), _ptr(bx), _ptr(by), _ptr(bz)))
        return U, bx, by, bz

    def nbors(self, ip):
        buf = np.zeros(self.np + 1, np.int32)
        k = lib().orc_num_nbors(self._h, ip, _ptr(buf))
        return buf[:k].copy()


# ---- cell-level entry points (unit pins) --------------------------------

def prim(u, faces, gamma):
    u, faces = _f64(u), _f64(faces)
    W = np.empty(8)
    lib().orc_prim(_ptr(u), _ptr(faces), gamma, _ptr(W))
    return W


def cfast(gamma, rho, p, bn, bt1, bt2):
    return lib().orc_cfast(gamma, rho, p, bn, bt1, bt2)


def mc(dl, dr):
    return lib().orc_mc(dl, dr)


def predict(W, dX, dY, dZ, gamma, h):
    W, dX, dY, dZ = (_f64(a) for a in (W, dX, dY, dZ))
    out = np.empty(8)
    lib().orc_predict(_ptr(W), _ptr(dX), _ptr(dY), _ptr(dZ), gamma, h, _ptr(out))
    return out


def hll(WL, WR, d, gamma):
    WL, WR = _f64(WL), _f64(WR)
    F = np.empty(7)
    S = np.empty(2)
    lib().orc_hll(_ptr(WL), _ptr(WR), d, gamma, _ptr(F), _ptr(S))
    return F, S


def hlld(WL, WR, d, gamma):
    WL, WR = _f64(WL), _f64(WR)
    F = np.empty(7)
    S = np.empty(2)
    lib().orc_hlld(_ptr(WL), _ptr(WR), d, gamma, _ptr(F), _ptr(S))
    return F, S


def hlld_fan(WL, WR, d, gamma):
    """(speeds S_L, S*_L, S_M, S*_R, S_R; states U*_L, U**_L, U**_R, U*_R in
    the normal frame: rho, rho u, rho v, rho w, E, By, Bz; the total pressure
    pT* of the fan), or None when the flux is a single side's."""
    WL, WR = _f64(WL), _f64(WR)
    fan = np.empty(34)
    if lib().orc_hlld_fan(_ptr(WL), _ptr(WR), d, gamma, _ptr(fan)):
        return None
    return fan[:5], fan[5:33].reshape(4, 7), float(fan[33])


def emf(Wll, Wrl, Wlr, Wrr, e, apa, ama, apb, amb):
    a = [_f64(x) for x in (Wll, Wrl, Wlr, Wrr)]
    return lib().orc_emf(*[_ptr(x) for x in a], e, apa, ama, apb, amb)


def pow2_floor(x):
    return lib().orc_pow2_floor(x)
