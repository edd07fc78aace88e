"""Thin ctypes binding of libdispatch_gpu.so (include/dispatch.h).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels.  The functions keep the C names; ``Dispatch`` bundles a context
handle with numpy (host) or torch (device) array marshalling.  If the library
cannot be loaded, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

DSP_OK = 0
DSP_ERR_INVALID_ARG = -1
DSP_ERR_OOM = -2
DSP_ERR_CUDA = -3
DSP_ERR_UNPHYSICAL = -4
DSP_ERR_TIMEOUT = -5
DSP_ERR_DEADLOCK = -6
DSP_ERR_SCHEDULE_OVERFLOW = -7
DSP_ERR_UNSUPPORTED = -8
DSP_ERR_BRACKET = -9
DSP_ERR_BOUNDS = -10

ERRORS = {v: k for k, v in globals().items() if k.startswith("DSP_ERR_")}

EXPORTS = ["dsp_create", "dsp_set_state", "dsp_advance", "dsp_get_state", "dsp_get_times",
           "dsp_get_schedule", "dsp_diagnostics", "dsp_save", "dsp_load", "dsp_last_error",
           "dsp_destroy", "dsp_diagnostics_noalloc", "dsp_autotune", "dsp_package_len", "dsp_pack", "dsp_unpack",
           "dsp_get_tuning"]

DSP_NOALLOC_MAX_PATCHES = 16384


class dsp_patch_desc(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("lo", ctypes.c_int64 * 3)]


class dsp_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("t0", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("grace", ctypes.c_double),
                ("box_lo", ctypes.c_double * 3), ("box_len", ctypes.c_double * 3),
                ("base_cells", ctypes.c_int32 * 3),
                ("nguard", ctypes.c_int32), ("nslices", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("time_mode", ctypes.c_int32), ("dt_pow2", ctypes.c_int32), ("dispatcher", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("tile_z", ctypes.c_int32),
                ("sched_capacity", ctypes.c_int64), ("timing", ctypes.c_int32), ("wait_budget", ctypes.c_int64),
                ("graph", ctypes.c_int32), ("variant", ctypes.c_int32), ("riemann", ctypes.c_int32),
                ("eta", ctypes.c_double), ("gamma_ad", ctypes.c_double), ("rho_i", ctypes.c_double),
                ("c_ohm", ctypes.c_double), ("c_ad", ctypes.c_double), ("time_order", ctypes.c_int32),
                ("owned", ctypes.c_void_p)]


class dsp_stats(ctypes.Structure):
    _fields_ = [("patch_updates", ctypes.c_int64), ("cell_updates", ctypes.c_int64),
                ("sweeps", ctypes.c_int64), ("fallbacks", ctypes.c_int64),
                ("t_min", ctypes.c_double), ("t_max", ctypes.c_double), ("status", ctypes.c_int32),
                ("kernel_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("plan_launches", ctypes.c_int64), ("floors", ctypes.c_int64)]


class dsp_sched_entry(ctypes.Structure):
    _fields_ = [("patch", ctypes.c_int64), ("t_start", ctypes.c_double), ("dt", ctypes.c_double)]


class dsp_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("mom", ctypes.c_double * 3), ("energy", ctypes.c_double),
                ("bmean", ctypes.c_double * 3), ("max_divb", ctypes.c_double), ("max_b", ctypes.c_double)]


_lock = threading.Lock()
_libs = {}
VP = ctypes.c_void_p


def lib_path(checked: bool = False) -> str:
    return _build.LIB_CHECKED if checked else _build.LIB


def load(build_if_missing: bool = True, checked: bool = False):
    """Load the CUDA library (building it in-tree with nvcc if needed); with
    checked=True the bounds-checked build (every global address of the
    update kernel tested, DSP_ERR_BOUNDS instead of a fault; three
    variants)."""
    with _lock:
        if checked in _libs:
            return _libs[checked]
        path = lib_path(checked)
        if build_if_missing and not _build.up_to_date(checked):
            _build.build(checked=checked)
        if not os.path.exists(path):
            raise RuntimeError("%s is not built; run paper_1705_10774_gb300.build" % path)
        L = ctypes.CDLL(path)
        L.dsp_create.argtypes = [ctypes.POINTER(dsp_patch_desc), ctypes.c_int32, ctypes.POINTER(dsp_params), VP,
                                 ctypes.POINTER(VP)]
        L.dsp_set_state.argtypes = [VP, ctypes.c_int32, ctypes.c_int32, VP, VP, VP, VP, ctypes.c_int32, ctypes.c_int32]
        L.dsp_advance.argtypes = [VP, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(dsp_stats)]
        L.dsp_get_state.argtypes = [VP, ctypes.c_int32, ctypes.c_int32, VP, VP, VP, VP, ctypes.c_int32, ctypes.c_int32]
        L.dsp_get_times.argtypes = [VP, VP, VP]
        L.dsp_get_schedule.argtypes = [VP, VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.dsp_diagnostics.argtypes = [VP, ctypes.POINTER(dsp_diag)]
        L.dsp_save.argtypes = [VP, VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        L.dsp_load.argtypes = [VP, VP, ctypes.c_size_t]
        L.dsp_last_error.argtypes = [VP]
        L.dsp_last_error.restype = ctypes.c_char_p
        L.dsp_destroy.argtypes = [VP]
        L.dsp_destroy.restype = None
        L.dsp_autotune.argtypes = [VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), VP, VP, ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_int32)]
        L.dsp_diagnostics_noalloc.argtypes = [VP, VP, VP, VP, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.c_double, VP,
                                              ctypes.POINTER(dsp_diag)]
        L.dsp_get_tuning.argtypes = [VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), VP, VP, VP]
        L.dsp_package_len.argtypes = [VP, VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
        L.dsp_pack.argtypes = [VP, VP, ctypes.c_int32, VP, VP, ctypes.c_int32]
        L.dsp_unpack.argtypes = [VP, VP, ctypes.c_int32, VP, VP, ctypes.c_int32]
        for name in EXPORTS:
            if name not in ("dsp_last_error", "dsp_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _libs[checked] = L
        return L


class DispatchError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "DSP_ERR"), code, msg))
        self.code = code


def _addr(a):
    """Device or host address of a torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), bool(a.is_cuda), (0 if str(a.dtype).endswith("float64") else 1)
    a = np.asarray(a)
    return a.ctypes.data_as(ctypes.c_void_p), False, (0 if a.dtype == np.float64 else 1)


class Dispatch:
    """A context of patches on a periodic box (level 0, optionally a level 1
    at half the cell size), on one GPU."""

    def __init__(self, n, lo, *, gamma, cfl, base_cells, box_len=(1.0, 1.0, 1.0), t0=0.0, dt_max=0.0,
                 nguard=3, nslices=3, precision=0, time_mode=0, dispatcher=1, tile_z=0,
                 sched_capacity=0, timing=0, wait_budget=0, graph=0, variant=-1, stream=None, level=None,
                 riemann=0, eta=0.0, gamma_ad=0.0, rho_i=1.0, c_ohm=0.1, c_ad=0.1, grace=0.0, time_order=1,
                 owned=None, checked=False):
        L = load(checked=checked)
        self._L = L
        n = np.asarray(n, dtype=np.int64).reshape(-1, 3)
        lo = np.asarray(lo, dtype=np.int64).reshape(-1, 3)
        self.np = n.shape[0]
        lev = np.zeros(self.np, np.int64) if level is None else np.asarray(level, np.int64).reshape(-1)
        descs = (dsp_patch_desc * self.np)()
        for i in range(self.np):
            descs[i].level = int(lev[i])
            for d in range(3):
                descs[i].n[d] = int(n[i, d])
                descs[i].lo[d] = int(lo[i, d])
        p = dsp_params()
        p.gamma, p.cfl, p.t0, p.dt_max, p.grace = gamma, cfl, t0, dt_max, grace
        for d in range(3):
            p.box_lo[d] = 0.0
            p.box_len[d] = box_len[d]
            p.base_cells[d] = int(base_cells[d])
        p.nguard, p.nslices, p.precision = nguard, nslices, precision
        p.time_mode, p.dt_pow2, p.dispatcher = time_mode, 1, dispatcher
        p.tile_x = p.tile_y = 0
        p.tile_z = tile_z
        p.sched_capacity = sched_capacity
        p.timing = timing
        p.wait_budget = wait_budget
        p.graph = graph
        p.variant = variant
        p.riemann = riemann
        # non-ideal MHD (Sec. 4.3): Ohmic resistivity, ambipolar drift
        # coefficient and ion density (0 turns a term off)
        p.eta, p.gamma_ad, p.rho_i, p.c_ohm, p.c_ad = eta, gamma_ad, rho_i, c_ohm, c_ad
        # grace of Eq. 1 and the order of the time inter- and extrapolation
        p.time_order = time_order
        # several processes (Sec. 3 C): 1 = owned, 0 = virtual copy
        own = None if owned is None else np.ascontiguousarray(owned, dtype=np.uint8).reshape(-1)
        if own is not None:
            assert own.size == self.np
            p.owned = own.ctypes.data_as(ctypes.c_void_p)
        self.params = p
        h = VP()
        rc = L.dsp_create(descs, self.np, ctypes.byref(p), VP(stream or 0), ctypes.byref(h))
        p.owned = None                            # read during dsp_create only
        if rc != 0:
            raise DispatchError(rc, "dsp_create rejected the layout or parameters")
        self._h = h
        self.n = n
        self.precision = precision
        nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
        per = np.stack([5 * nx * ny * nz, (nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1)], axis=1)
        self.per_patch = per                      # (np, 4) values of U, bx, by, bz per patch
        self.sizes = tuple(int(x) for x in per.sum(axis=0))

    def _check(self, rc):
        if rc != 0 and rc != DSP_ERR_SCHEDULE_OVERFLOW:
            raise DispatchError(rc, self._L.dsp_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._L.dsp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, U, bx, by, bz, first=0, count=None):
        count = self.np - first if count is None else count
        ptrs = [_addr(a) for a in (U, bx, by, bz)]
        dev, dt = ptrs[0][1], ptrs[0][2]
        assert all(p[1] == dev and p[2] == dt for p in ptrs)
        self._check(self._L.dsp_set_state(self._h, first, count, *[p[0] for p in ptrs], dt, int(dev)))

    def get_state(self, out=None, dtype=np.float64, first=0, count=None):
        count = self.np - first if count is None else count
        if out is None:
            sz = self.per_patch[first:first + count].sum(axis=0)
            out = [np.empty(int(s), dtype=dtype) for s in sz]
        ptrs = [_addr(a) for a in out]
        self._check(self._L.dsp_get_state(self._h, first, count, *[p[0] for p in ptrs], ptrs[0][2], int(ptrs[0][1])))
        return out

    def advance(self, t_end=float("inf"), max_sweeps=0):
        st = dsp_stats()
        self._check(self._L.dsp_advance(self._h, t_end, max_sweeps, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in dsp_stats._fields_}

    def times(self):
        t = np.empty(self.np)
        dt = np.empty(self.np)
        self._check(self._L.dsp_get_times(self._h, t.ctypes.data_as(VP), dt.ctypes.data_as(VP)))
        return t, dt

    def schedule(self):
        n = ctypes.c_int64()
        self._L.dsp_get_schedule(self._h, None, 0, ctypes.byref(n))
        cap = n.value
        buf = (dsp_sched_entry * max(cap, 1))()
        rc = self._check(self._L.dsp_get_schedule(self._h, buf, cap, ctypes.byref(n)))
        k = min(cap, n.value)
        a = np.frombuffer(buf, dtype=np.dtype([("patch", np.int64), ("t", np.float64), ("dt", np.float64)]),
                          count=k).copy() if k else np.zeros(0, dtype=[("patch", np.int64), ("t", np.float64), ("dt", np.float64)])
        if rc == DSP_ERR_SCHEDULE_OVERFLOW:
            raise DispatchError(rc, "schedule log overflowed")
        return a["patch"], a["t"], a["dt"]

    def diagnostics(self):
        d = dsp_diag()
        self._check(self._L.dsp_diagnostics(self._h, ctypes.byref(d)))
        return dict(mass=d.mass, mom=np.array(d.mom[:]), energy=d.energy, bmean=np.array(d.bmean[:]),
                    max_divb=d.max_divb, max_b=d.max_b)

    def autotune(self, reps=3):
        """dsp_autotune: returns (variant chosen for size class 0,
        {variant id: ms per launch} of class 0's whole-height candidates);
        tuning() and self.tuning_log give every class's choice and
        candidates."""
        chosen = ctypes.c_int32()
        n = ctypes.c_int32()
        cap = 256
        ms = np.zeros(cap)
        ids = np.zeros(cap, np.int32)
        self._check(self._L.dsp_autotune(self._h, reps, ctypes.byref(chosen), ms.ctypes.data_as(VP),
                                        ids.ctypes.data_as(VP), cap, ctypes.byref(n)))
        k = min(n.value, cap)
        self.tuning_log = [dict(cls=int(i) // 1000000, tile_z=(int(i) // 1000) % 1000, variant=int(i) % 1000,
                                ms=float(m)) for i, m in zip(ids[:k], ms[:k])]
        first = {}
        for e in self.tuning_log:
            if e["cls"] == 0:
                first.setdefault(e["variant"], e["ms"])
        return chosen.value, first

    def tuning(self):
        """dsp_get_tuning: [{size, variant, tile_z}] per size class."""
        nc = ctypes.c_int32()
        sizes = np.zeros(12, np.int32)
        var = np.zeros(4, np.int32)
        tz = np.zeros(4, np.int32)
        self._check(self._L.dsp_get_tuning(self._h, 4, ctypes.byref(nc), sizes.ctypes.data_as(VP),
                                          var.ctypes.data_as(VP), tz.ctypes.data_as(VP)))
        return [dict(size=sizes[3 * k:3 * k + 3].tolist(), variant=int(var[k]), tile_z=int(tz[k]))
                for k in range(min(nc.value, 4))]

    def save(self) -> bytes:
        used = ctypes.c_size_t()
        self._check(self._L.dsp_save(self._h, None, 0, ctypes.byref(used)))
        buf = ctypes.create_string_buffer(used.value)
        self._check(self._L.dsp_save(self._h, buf, used.value, ctypes.byref(used)))
        return buf.raw

    def save_array(self) -> np.ndarray:
        """dsp_save into a numpy byte array (no second copy of a large state)."""
        used = ctypes.c_size_t()
        self._check(self._L.dsp_save(self._h, None, 0, ctypes.byref(used)))
        buf = np.empty(used.value, np.uint8)
        self._check(self._L.dsp_save(self._h, buf.ctypes.data_as(ctypes.c_void_p), used.value, ctypes.byref(used)))
        return buf

    def load_state(self, blob: bytes):
        self._check(self._L.dsp_load(self._h, blob, len(blob)))

    # ---- packages between processes (Sec. 3 C)
    def package_len(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        n = ctypes.c_int64()
        self._check(self._L.dsp_package_len(self._h, ids.ctypes.data_as(VP), ids.size, ctypes.byref(n)))
        return n.value

    def pack(self, ids, device=True):
        """The packages of the listed patches: (values, meta (k, 3)), as torch
        CUDA tensors (device=True) or numpy arrays."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        n = self.package_len(ids)
        if device:
            import torch
            dt = torch.float32 if self.precision == 1 else torch.float64
            buf = torch.empty(max(n, 1), dtype=dt, device="cuda")
            meta = torch.empty((max(ids.size, 1), 3), dtype=torch.float64, device="cuda")
            self._check(self._L.dsp_pack(self._h, ids.ctypes.data_as(VP), ids.size, VP(buf.data_ptr()),
                                        VP(meta.data_ptr()), 1))
            return buf[:n], meta[:ids.size]
        buf = np.empty(max(n, 1), np.float32 if self.precision == 1 else np.float64)
        meta = np.empty((max(ids.size, 1), 3))
        self._check(self._L.dsp_pack(self._h, ids.ctypes.data_as(VP), ids.size, buf.ctypes.data_as(VP),
                                    meta.ctypes.data_as(VP), 0))
        return buf[:n], meta[:ids.size]

    def unpack(self, ids, buf, meta):
        """Store received packages as the newest slices of the listed virtual
        patches (torch CUDA tensors or numpy arrays, both of one kind)."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        if ids.size == 0:
            return
        if not hasattr(buf, "data_ptr"):
            buf = np.ascontiguousarray(buf)
            meta = np.ascontiguousarray(meta, dtype=np.float64)
        b, bdev, _ = _addr(buf)
        m, mdev, _ = _addr(meta)
        assert bdev == mdev
        self._check(self._L.dsp_unpack(self._h, ids.ctypes.data_as(VP), ids.size, b, m, int(bdev)))


def _check_noalloc_arrays(arrays, npatch, n):
    """The checks dsp_diagnostics_noalloc cannot make on raw pointers: four
    contiguous CUDA tensors on the current device, one dtype (float64 or
    float32), each holding exactly npatch patches of n[0] x n[1] x n[2] cells
    in the dsp_set_state layout.  Raises ValueError before anything reaches
    the device."""
    if len(arrays) != 4:
        raise ValueError("expected U, bx, by, bz")
    nx, ny, nz = (int(x) for x in n)
    if npatch < 0 or min(nx, ny, nz) < 1:
        raise ValueError("npatch must be >= 0 and every n >= 1")
    want = [npatch * 5 * nx * ny * nz, npatch * (nx + 1) * ny * nz, npatch * nx * (ny + 1) * nz,
            npatch * nx * ny * (nz + 1)]
    dtypes = set()
    for name, a, w in zip(("U", "bx", "by", "bz"), arrays, want):
        if not (hasattr(a, "is_cuda") and hasattr(a, "data_ptr")):
            raise ValueError("%s must be a torch CUDA tensor (got %s)" % (name, type(a).__name__))
        if not a.is_cuda:
            raise ValueError("%s must be on a CUDA device" % name)
        import torch
        if a.device.index != torch.cuda.current_device():
            raise ValueError("%s is on cuda:%s, not the current device" % (name, a.device.index))
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if a.numel() != w:
            raise ValueError("%s holds %d values, expected %d for %d patches of %s cells"
                             % (name, a.numel(), w, npatch, (nx, ny, nz)))
        dtypes.add(str(a.dtype))
    if len(dtypes) != 1 or dtypes.pop() not in ("torch.float64", "torch.float32"):
        raise ValueError("U, bx, by, bz must share one dtype, float64 or float32")


def diagnostics_noalloc(U, bx, by, bz, npatch, n, dx, stream=None):
    """dsp_diagnostics_noalloc on caller-owned device arrays (torch CUDA
    tensors in the dsp_set_state layout, all patches of n cells and cell
    size dx): the library allocates nothing.  The arrays are checked first
    (ValueError); the library checks npatch against its limit and dx."""
    _check_noalloc_arrays((U, bx, by, bz), int(npatch), n)
    L = load()
    ptrs = [_addr(a) for a in (U, bx, by, bz)]
    dt = ptrs[0][2]
    nn = (ctypes.c_int32 * 3)(*[int(x) for x in n])
    d = dsp_diag()
    rc = L.dsp_diagnostics_noalloc(*[p[0] for p in ptrs], dt, int(npatch), nn, float(dx), VP(stream or 0),
                                   ctypes.byref(d))
    if rc != 0:
        raise DispatchError(rc, "dsp_diagnostics_noalloc failed")
    return dict(mass=d.mass, mom=np.array(d.mom[:]), energy=d.energy, bmean=np.array(d.bmean[:]),
                max_divb=d.max_divb, max_b=d.max_b)
