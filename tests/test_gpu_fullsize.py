"""Parity at full benchmark sizes, on outputs the oracle can compute one by
one: the GPU runs the whole workload in the benchmark's launch configuration,
the oracle loads the GPU's state at some point and reproduces the next update
of sampled patches (and the step and ready set of that sweep)."""
import json
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import Dispatch
from oracle import Oracle

from fields import NAMES, field_errors

TOL64 = 1e-11


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def patch_slices(lay, arrays, P):
    n = lay.n[0]
    nc = int(n[0] * n[1] * n[2])
    sizes = [5 * nc, (n[0] + 1) * n[1] * n[2], n[0] * (n[1] + 1) * n[2], n[0] * n[1] * (n[2] + 1)]
    return [a[P * s:(P + 1) * s] for a, s in zip(arrays, sizes)]


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("opts", [{}, dict(riemann=1), dict(eta=1e-4, gamma_ad=75.0, rho_i=1.0)],
                         ids=["hll", "hlld", "nonideal"])
def test_turbulence_256cubed_sampled_patches_fp64(precision, opts):
    """512 patches of 32^3, global steps, both FP64 builds, in each of the
    benchmark's forms (HLL, HLLD faces, non-ideal terms): after 3 steps the
    oracle takes the GPU state, recomputes the global step and the 4th update
    of 8 patches."""
    lay, f = ics.config_turbulence(seed=10774, patches=8, n=32, mach=2.0)
    state = ics.to_patches(lay, f)
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, **opts)
    g = Dispatch(lay.n, lay.lo, time_mode=0, precision=precision, **kw)
    g.set_state(*[torch.from_numpy(a).cuda() for a in state])
    g.advance(max_sweeps=3)
    snap = g.get_state()
    t3 = g.times()[0]
    assert np.all(t3 == t3[0])
    g.advance(max_sweeps=1)
    after = g.get_state()
    t4, dt4 = g.times()
    o = Oracle(lay.n, lay.lo, t0=float(t3[0]), **kw)
    o.set_state(*snap)
    dt = min(o.patch_dt(i) for i in range(lay.npatch))
    assert np.all(dt4 == dt) and np.all(t4 == t3[0] + dt)
    for P in (0, 7, 63, 64, 200, 365, 448, 511):
        ref = o.update_patch(P, dt)[:4]
        got = patch_slices(lay, after, P)
        errs = field_errors(got, ref, [int(np.prod(lay.n[P]))])
        assert max(errs.values()) <= TOL64, (P, errs)


@pytest.mark.parametrize("opts", [{}, dict(riemann=1), dict(eta=1e-4, gamma_ad=75.0, rho_i=1.0)],
                         ids=["hll", "hlld", "nonideal"])
def test_turbulence_256cubed_sampled_patches_fp32(opts):
    """The benchmark's FP32 forms (autotuned, global steps) at full size:
    after 3 steps the oracle takes the GPU's FP32 state (exactly, in FP64)
    and recomputes the 4th update of 8 patches with the GPU's step, within
    1e-5 of each patch's largest value; the step is the oracle's (the FP32
    signal speeds may move it across a power of two only in rare ties)."""
    lay, f = ics.config_turbulence(seed=10774, patches=8, n=32, mach=2.0)
    state = ics.to_patches(lay, f)
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, **opts)
    g = Dispatch(lay.n, lay.lo, time_mode=0, precision=1, **kw)
    g.set_state(*[torch.from_numpy(a).float().cuda() for a in state])
    g.autotune(reps=1)
    g.advance(max_sweeps=3)
    snap = g.get_state()
    t3 = g.times()[0]
    g.advance(max_sweeps=1)
    after = g.get_state()
    t4, dt4 = g.times()
    dt = float(dt4[0])
    o = Oracle(lay.n, lay.lo, t0=float(t3[0]), **kw)
    o.set_state(*snap)
    assert min(o.patch_dt(i) for i in range(lay.npatch)) == dt
    for P in (0, 7, 63, 64, 200, 365, 448, 511):
        ref = o.update_patch(P, dt)[:4]
        got = patch_slices(lay, after, P)
        scale = max(float(np.max(np.abs(b))) for b in ref)
        for a, b in zip(got, ref):
            assert float(np.max(np.abs(a - b))) <= 1e-5 * scale


def parse_save(blob, lay, nslot):
    magic = blob[:8]
    assert magic.startswith(b"DSPSAVE")
    version, npch, ns, prec = struct.unpack_from("<4i", blob, 8)
    _, slot_stride = struct.unpack_from("<2q", blob, 24)
    off = 40
    ts = np.frombuffer(blob, np.float64, npch * ns, off).reshape(npch, ns); off += 8 * npch * ns
    sm = np.frombuffer(blob, np.float64, npch * ns, off).reshape(npch, ns); off += 8 * npch * ns
    latest = np.frombuffer(blob, np.int32, npch, off); off += 4 * npch
    dtl = np.frombuffer(blob, np.float64, npch, off); off += 8 * npch
    # slices are stored slice-major; these patches all have the same size
    slab = np.frombuffer(blob, np.float64, ns * slot_stride, off).reshape(ns, npch, slot_stride // npch)
    return ts, sm, latest, dtl, slab


def test_local_steps_4096_patches_sampled_sweep_fp64():
    """4096 patches of 16^3 with local steps (log-normal density, hot
    sphere): after 24 sweeps the oracle loads the GPU's full dispatcher state
    (every slice), finds the ready set and steps of the next sweep, and
    reproduces sampled updates of it."""
    lay, f = ics.config_lts(patches=16, n=16)
    state = ics.to_patches(lay, f)
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    t_end = 0.05
    g = Dispatch(lay.n, lay.lo, time_mode=1, sched_capacity=1 << 22, **kw)
    g.set_state(*[torch.from_numpy(a).cuda() for a in state])
    g.advance(t_end=t_end, max_sweeps=24)
    blob = g.save()
    n_before = len(g.schedule()[0])
    g.advance(t_end=t_end, max_sweeps=1)
    sp, st, sdt = g.schedule()
    sp, st, sdt = sp[n_before:], st[n_before:], sdt[n_before:]
    after = g.get_state()
    ts, sm, latest, dtl, slab = parse_save(blob, lay, 3)
    o = Oracle(lay.n, lay.lo, time_mode=1, **kw)
    n = lay.n[0]
    nc = int(n[0] * n[1] * n[2])
    cuts = np.cumsum([5 * nc, (n[0] + 1) * n[1] * n[2], n[0] * (n[1] + 1) * n[2]])
    for P in range(lay.npatch):
        for s in range(3):
            U, bx, by, bz = np.split(slab[s, P], cuts)
            o.set_slot(P, s, float(ts[P, s]), U, bx, by, bz)
        o.set_latest(P, int(latest[P]), float(dtl[P]))
    t = ts[np.arange(lay.npatch), latest]
    ready = []
    for P in range(lay.npatch):
        if t[P] < t_end and all(t[P] <= t[q] for q in o.nbors(P)):
            ready.append(P)
    assert sorted(sp.tolist()) == ready
    assert len(np.unique(dtl[dtl > 0])) >= 2 or len(np.unique(sdt)) >= 2
    want = {P: o.patch_dt(P, t_end) for P in ready}
    for P, t0, d in zip(sp, st, sdt):
        assert t0 == t[P] and d == want[int(P)]
    rng = np.random.default_rng(0)
    for P in rng.choice(ready, size=min(6, len(ready)), replace=False):
        ref = o.update_patch(int(P), want[int(P)])[:4]
        got = patch_slices(lay, after, int(P))
        errs = field_errors(got, ref, [int(np.prod(lay.n[int(P)]))])
        assert max(errs.values()) <= TOL64, (P, errs)


def test_fp64_fma_build_after_100_steps_of_the_benchmark():
    """The benchmark's 100 global steps of the 256^3 workload with both FP64
    builds: the FMA-free build equals the oracle bit for bit (pinned above and
    in the parity tests), so its result stands for the oracle's; the FMA build
    must stay within 1e-11 relative L-infinity per field, with the same
    steps; the FP32 form within 1e-5 relative L1 per field (density, the
    momentum components, energy, the three face fields)."""
    lay, f = ics.config_turbulence(seed=10774, patches=8, n=32, mach=2.0)
    state = [torch.from_numpy(a).cuda() for a in ics.to_patches(lay, f)]
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=0)
    res = []
    for prec in (0, 2):
        g = Dispatch(lay.n, lay.lo, precision=prec, **kw)
        g.set_state(*state)
        g.advance(max_sweeps=100)
        res.append((g.get_state(), g.times()))
        g.close()
    (a, ta), (b, tb) = res
    assert np.array_equal(ta[0], tb[0]) and np.array_equal(ta[1], tb[1])
    errs = field_errors(b, a, np.prod(lay.n, axis=1))
    assert max(errs.values()) <= TOL64, errs
    g = Dispatch(lay.n, lay.lo, precision=1, **kw)
    g.set_state(*[x.float() for x in state])
    g.advance(max_sweeps=100)
    c = g.get_state()
    g.close()
    A = a[0].reshape(lay.npatch, 5, -1)
    C = c[0].reshape(lay.npatch, 5, -1)
    fields = [(A[:, k], C[:, k]) for k in range(5)] + list(zip(a[1:], c[1:]))
    rel = {n: float(np.abs(x - y).sum() / np.abs(x).sum()) for n, (x, y) in zip(NAMES, fields)}
    print("FP32_PER_FIELD turbulence 256^3, 100 steps, relative L1: %s" % json.dumps(rel))
    for n, e in rel.items():
        assert e <= 1e-5, (n, e)


@pytest.mark.parametrize("precision", [2, 1])
def test_local_steps_4096_patches_queue_equals_sweeps(precision):
    """The full local-step input with both dispatchers: the persistent ready
    queue (thousands of patches in flight in one launch) and the sweeps give
    the same schedule as a set and the same state bit for bit."""
    lay, f = ics.config_lts(patches=16, n=16)
    state = [torch.from_numpy(a).cuda() for a in ics.to_patches(lay, f)]
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1,
              precision=precision, sched_capacity=1 << 22)
    t_end = 0.004
    out = []
    for disp in (0, 1):
        g = Dispatch(lay.n, lay.lo, dispatcher=disp, **kw)
        g.set_state(*state)
        st = g.advance(t_end=t_end)
        out.append((g.get_state(), sorted(zip(*(x.tolist() for x in g.schedule()))), st))
        g.close()
    (a, sa, st_q), (b, sb, st_s) = out
    assert sa == sb
    assert st_q["cell_updates"] == st_s["cell_updates"]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def parse_save_any(blob):
    """Times, signal speeds, newest-slot indices, last steps and the slab
    (slice-major, any patch sizes) of a dsp_save blob."""
    assert bytes(blob[:8]).startswith(b"DSPSAVE")
    version, npch, ns, prec = struct.unpack_from("<4i", blob, 8)
    _, slot_stride = struct.unpack_from("<2q", blob, 24)
    off = 40
    ts = np.frombuffer(blob, np.float64, npch * ns, off).reshape(npch, ns); off += 8 * npch * ns
    sm = np.frombuffer(blob, np.float64, npch * ns, off).reshape(npch, ns); off += 8 * npch * ns
    latest = np.frombuffer(blob, np.int32, npch, off); off += 4 * npch
    dtl = np.frombuffer(blob, np.float64, npch, off); off += 8 * npch
    dt = np.float32 if prec == 1 else np.float64
    slab = np.frombuffer(blob, dt, ns * slot_stride, off).reshape(ns, slot_stride)
    return ts, latest, dtl, slab


def _patch_lengths(n):
    n = n.astype(np.int64)
    nc = n[:, 0] * n[:, 1] * n[:, 2]
    parts = np.stack([5 * nc, (n[:, 0] + 1) * n[:, 1] * n[:, 2], n[:, 0] * (n[:, 1] + 1) * n[:, 2],
                      n[:, 0] * n[:, 1] * (n[:, 2] + 1)], axis=1)
    return parts, np.concatenate([[0], np.cumsum(parts.sum(axis=1))])


def _around(lay, P, margin):
    """Patches whose box meets patch P's box widened by `margin` level-0
    cells (periodic), in level-1 cell units: a superset of P's neighbours."""
    s = (2 // 2 ** lay.levels)[:, None]
    lo, hi = lay.lo * s, (lay.lo + lay.n) * s
    L = 2 * np.array(lay.base_cells)
    a, b = lo[P] - 2 * margin, hi[P] + 2 * margin
    hit = np.ones(lay.npatch, bool)
    for d in range(3):
        ax = np.zeros(lay.npatch, bool)
        for sh in (-L[d], 0, L[d]):
            ax |= (lo[:, d] + sh < b[d]) & (hi[:, d] + sh > a[d])
        hit &= ax
    return np.flatnonzero(hit)


def test_two_levels_full_size_sampled_updates_fp32():
    """The uneven two-level solve at full size (8.3k patches of 16^3 / 24^3 /
    32^3, 1.5e8 cells) in the benchmark's launch configuration (FP32 state,
    local steps, sweeps replayed from CUDA graphs, autotuned).  After 32
    sweeps the oracle takes the GPU's slices around sampled ready patches --
    level-1 patches at the edge of the refined region (prolonged guards) and
    level-0 patches next to or under it (restricted guards) -- and reproduces
    their steps and their next updates in FP64 from the same FP32 inputs."""
    lay, arrays = ics.config_two_level(5)
    kw = dict(gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    g = Dispatch(lay.n, lay.lo, level=lay.levels, time_mode=1, precision=1, graph=1, sched_capacity=1 << 22, **kw)
    g.set_state(*[torch.from_numpy(a).cuda() for a in arrays])
    del arrays
    g.autotune(reps=1)
    g.advance(t_end=1.0, max_sweeps=32)
    parts, offs = _patch_lengths(lay.n)
    X = lay.base_cells[0]
    r1 = (2 * (3 * X // 8), 2 * (5 * X // 8))        # refined region in level-1 cells
    s = (2 // 2 ** lay.levels)[:, None]
    lo1, hi1 = lay.lo * s, (lay.lo + lay.n) * s
    edge_fine = (lay.levels == 1) & np.any((lo1 == r1[0]) | (hi1 == r1[1]), axis=1)
    near = np.all((hi1 > r1[0] - 8) & (lo1 < r1[1] + 8), axis=1)
    coarse_near = (lay.levels == 0) & near
    seen = {"fine": 0, "coarse": 0}
    rng = np.random.default_rng(1)
    for _ in range(4):
        blob = g.save_array()
        n_before = len(g.schedule()[0])
        g.advance(t_end=1.0, max_sweeps=1)
        sp, st_, sdt = (x[n_before:] for x in g.schedule())
        ts, latest, dtl, slab = parse_save_any(blob)
        picks = []
        for name, mask in (("fine", edge_fine), ("coarse", coarse_near)):
            cand = [int(P) for P in sp if mask[P]]
            picks += [(name, P) for P in rng.permutation(cand)[:2]]
        for name, P in picks:
            S = _around(lay, P, 6)
            o = Oracle(lay.n[S], lay.lo[S], level=lay.levels[S], time_mode=1, **kw)
            for k, Q in enumerate(S):
                for sl in range(3):
                    seg = slab[sl, offs[Q]:offs[Q + 1]].astype(np.float64)
                    U, bx, by, bz = np.split(seg, np.cumsum(parts[Q])[:3])
                    o.set_slot(k, sl, float(ts[Q, sl]), U, bx, by, bz)
                o.set_latest(k, int(latest[Q]), float(dtl[Q]))
            k = int(np.flatnonzero(S == P)[0])
            j = int(np.flatnonzero(sp == P)[0])
            assert st_[j] == ts[P, latest[P]]
            assert o.patch_dt(k, 1.0) == sdt[j]
            ref = o.update_patch(k, float(sdt[j]))[:4]
            got = g.get_state(first=P, count=1)
            scale = max(float(np.max(np.abs(b))) for b in ref)
            for a, b in zip(got, ref):
                assert float(np.max(np.abs(a - b))) <= 1e-5 * scale, (name, P)
            seen[name] += 1
        del blob, slab
        if seen["fine"] >= 2 and seen["coarse"] >= 2:
            break
    assert seen["fine"] >= 2 and seen["coarse"] >= 2, seen


def test_largest_box_1024cubed_fp32_sampled_first_step():
    """The largest box the tests run: 1024^3 cells as 32^3 patches of 32^3
    in FP32 (3 slices, 104 GB on the device; slice offsets of the later
    patches exceed 2^32 elements).  One global step from a smooth analytic
    state uploaded in chunks; the oracle reproduces the updates of patches at
    both ends of the patch range from the same FP32 initial values."""
    lay = ics.cartesian(32, 32)
    # separable smooth fields (cheap to sample: 1-D factors broadcast); each
    # face component is independent of its own normal coordinate, so the
    # discrete divergence is exactly zero
    tp = 2 * np.pi
    X1 = lambda x: x[:1, :1, :]
    Y1 = lambda y: y[:1, :, :1]
    Z1 = lambda z: z[:, :1, :1]
    rho = lambda x, y, z: 1.0 + 0.2 * np.sin(tp * X1(x) + 0.3) * np.sin(tp * Z1(z) + 1.1)
    vel = lambda x, y, z: (0.5 * np.sin(tp * Y1(y) + 0.7) * np.cos(tp * Z1(z)), 0.4 * np.sin(2 * tp * X1(x) + 0.2),
                           0.3 * np.cos(tp * X1(x)) * np.sin(tp * Y1(y) + 1.9))
    pre = lambda x, y, z: 0.6 + 0 * X1(x)
    faces = (lambda x, y, z: 0.8 + 0.05 * np.sin(tp * Y1(y)) * np.cos(tp * Z1(z)),
             lambda x, y, z: 0.05 * np.sin(tp * Z1(z) + 0.4) + 0 * X1(x),
             lambda x, y, z: 0.05 * np.cos(tp * X1(x) + 0.9) * np.sin(tp * Y1(y)))

    def arrays(ids):
        sub = ics.Layout(n=lay.n[ids], lo=lay.lo[ids], base_cells=lay.base_cells, box_len=lay.box_len)
        return ics.patches_from_functions(sub, rho, vel, pre, 5.0 / 3.0, faces=faces, dtype=np.float32)

    kw = dict(gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    g = Dispatch(lay.n, lay.lo, time_mode=0, precision=1, **kw)
    chunk = 1024
    for first in range(0, lay.npatch, chunk):
        ids = np.arange(first, min(first + chunk, lay.npatch))
        g.set_state(*[torch.from_numpy(a).cuda() for a in arrays(ids)], first=first, count=len(ids))
    st = g.advance(max_sweeps=1)
    assert st["cell_updates"] == 1024 ** 3
    t, dt = g.times()
    assert np.all(dt == dt[0]) and dt[0] > 0
    for P in (0, 1023, 16400, lay.npatch - 1):
        S = _around(lay, P, 4)
        o = Oracle(lay.n[S], lay.lo[S], time_mode=0, **kw)
        o.set_state(*[a.astype(np.float64) for a in arrays(S)])
        kP = int(np.flatnonzero(S == P)[0])
        ref = o.update_patch(kP, float(dt[0]))[:4]
        got = g.get_state(first=P, count=1)
        scale = max(float(np.max(np.abs(b))) for b in ref)
        for a, b in zip(got, ref):
            assert float(np.max(np.abs(a - b))) <= 1e-5 * scale, P
    g.close()
