#!/usr/bin/env python
"""Benchmark of the per-patch update: MHD cell-updates/s on one GB300.

Workload of the benchmark line: the 3-D Orszag-Tang vortex on a periodic
512^3 box cut into 16^3 = 4096 patches of 32^3 cells (rho = 25/(36 pi),
p = 5/(12 pi), v = (-sin 2 pi y, sin 2 pi x, 0), b from A_z, a seeded 1e-3
random v_z), one global power-of-two Courant step per sweep (C = 0.4).  A
bench "step" is one sweep: every patch fills its guard zones, advances one
step and publishes it.  `value` is the FP64 form (fused multiply-adds,
checked against the FP64 oracle to 1e-11 per field); `value_f32` and
`forms.f32` the FP32-state form of the same run.  A slice (8.7 GB in FP64)
is far larger than L2, so no flush is needed between steps.  Side forms on
the 256^3 decaying-turbulence input (512 patches of 32^3): the FMA-free FP64
build, HLLD faces and the non-ideal terms, in both precisions.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (32 patch updates of the 512^3 input per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MHD cell-updates/s (FP64 vs FP32 form) and % of GB300 HBM roofline"
UNIT = "cell-updates/s"
# the benchmark line: 16^3 patches of 32^3 (512^3); the side forms: 8^3 (256^3)
PATCHES, NCELL = 16, 32
SIDE_PATCHES = 8
HBM_FALLBACK_GBS = 6800.0


def workload(patches=PATCHES):
    L = patches * NCELL
    return ("Orszag-Tang vortex, %d^3 periodic, %d patches of 32^3, global dt, CFL 0.4" % (L, patches ** 3))


SIDE_WORKLOAD = "decaying MHD turbulence, 256^3 periodic, 512 patches of 32^3, global dt, CFL 0.4"
# the timed FP64 form: FP64 state and arithmetic with fused multiply-adds
# (checked against the FP64 oracle to 1e-11); the FMA-free build that matches
# the oracle bit for bit is timed too and reported as forms.f64_exact
F64_PRECISION = 2
# coefficients of the non-ideal forms: Ohmic resistivity, and the C-shock
# experiment's ambipolar drift coefficient and ion density (Sec. 5.4)
NONIDEAL = dict(eta=1e-4, gamma_ad=75.0, rho_i=1.0)

# DRAM bytes (read + write) per cell-update of the update kernel, by
# compiled variant, from ncu's dram__bytes_read.sum + dram__bytes_write.sum
# of one launch divided by the cells it updated (captures of smaller cases
# of the same kernel: traffic grows in proportion to the cells); a variant
# without an entry reports null.
TRAFFIC_PER_CELL = {4: (555.389952e6 + 432.454656e6) / 7077888, 5: (237.726720e6 + 193.273088e6) / 7077888,
                    10: (542.026496e6 + 422.849280e6) / 7077888, 15: (527.585792e6 + 424.571136e6) / 7077888}


def guard_fraction(n, g):
    """Guard cells per interior cell of an n^3 patch with g guard layers."""
    return ((n + 2 * g) ** 3 - n ** 3) / n ** 3


def alg_bytes_per_cell(n, esize, sbar=1.0, g=3):
    """Algorithmic HBM bytes per cell-update: read and write the 8 stored
    fields once, plus the guard shell of g layers taken from sbar neighbour
    slices (g = 3 as the guard zones are specified; the stencil itself reads
    g = 2, which alg_bytes_radius2 gives)."""
    V = 8
    return esize * (2 * V + sbar * guard_fraction(n, g) * V)


def alg_bytes_radius2(n, esize, sbar=1.0):
    return alg_bytes_per_cell(n, esize, sbar, g=2)


# Algorithmic floating-point operations per cell-update (add, subtract,
# multiply, divide and square root count one each; min, max, abs and compares
# count none), from the per-cell arithmetic of the step as defined: primitive
# recovery; 21 MC-limited slopes (two differences each) and 3 face
# differences for the normal field; the Hancock predictor; its positivity
# test; 3 faces of left and right states (8 components each); 3 HLL fluxes
# (5 components, subsonic branch); 3 edge EMFs from 4 corner states of 4
# components each; the conservative and constrained-transport update; the
# signal speed of the new state.  Guard-zone interpolation is not counted
# (global steps copy neighbour slices).
ALG_FLOPS = {"primitives": 28, "slopes": 21 * 7 + 3, "predictor": 130, "positivity": 18, "face_states": 3 * 32,
             "hll": 3 * 176, "edge_emf": 3 * 111, "update": 5 * 7 + 3 * 5, "signal_speed": 28 + 63}
ALG_FLOPS_PER_CELL = sum(ALG_FLOPS.values())
# With HLLD faces (double-star branch, both star states regular), each face
# replaces the 37 flops of the HLL blend (5 components and the reciprocal of
# SR - SL) by 170: the contact speed and total pressure (20), per side the
# star density, velocity, field and energy and sqrt(rho*) (2 x 34, plus Bn^2),
# and the double-star states, their energy and the flux of the region (81).
ALG_FLOPS_HLLD = dict(ALG_FLOPS, hll=0, hlld=3 * (176 - 37 + 170))
ALG_FLOPS_PER_CELL_HLLD = sum(ALG_FLOPS_HLLD.values())

# Arithmetic peaks derived from unit counts and the maximum SM clock:
# 152 SMs at 2.07 GHz; FP64: 2 fused multiply-adds per SM per cycle (the
# GB300 FP64 rate, 1.26 TFLOP/s); FP32: 128 lanes per SM.
SMS, SM_GHZ = 152, 2.07
FP64_PEAK_TFLOPS = SMS * 2 * 2 * SM_GHZ / 1e3
FP32_PEAK_TFLOPS = SMS * 128 * 2 * SM_GHZ / 1e3


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as fh:
                d = json.load(fh)
            v = d.get("hbm_gbs") or d.get("hbm_GBs") or d.get("hbm")
            if isinstance(v, dict):
                v = v.get("value")
            if v:
                return float(v), "measured"
        except Exception:
            pass
    return HBM_FALLBACK_GBS, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
        return tdist, rank, ws
    return None, rank, ws


def max_over_ranks(td, x):
    if td is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(td, x):
    if td is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    td.all_reduce(t, op=td.ReduceOp.SUM)
    return float(t.item())


def make_input(patches=PATCHES):
    """The benchmark line's input: Orszag-Tang patch arrays (FP64, host)."""
    from paper_1705_10774_gb300 import ics
    return ics.orszag_tang_patches(seed=10775, patches=patches, n=NCELL)


def make_side_input(patches=SIDE_PATCHES):
    from paper_1705_10774_gb300 import ics
    lay, f = ics.config_turbulence(seed=10774, patches=patches, n=NCELL, mach=2.0)
    return lay, ics.to_patches(lay, f)


def rooflines(ncells, esize, kernel_ms, hbm_peak, peak_kind, flops_per_cell=ALG_FLOPS_PER_CELL):
    """The update kernel against its two roofs: HBM bandwidth (algorithmic
    bytes) and arithmetic (algorithmic flops against the FP64 or FP32 peak).
    The bound named first is the one the kernel is limited by (FP64: the
    FP64 pipe; FP32: neither, it is issue-bound, and the HBM figure is the
    benchmark's metric)."""
    bpl = alg_bytes_per_cell(NCELL, esize) * ncells
    gbs = bpl / (kernel_ms * 1e-3) / 1e9
    fpl = flops_per_cell * ncells
    tfs = fpl / (kernel_ms * 1e-3) / 1e12
    fpeak = FP64_PEAK_TFLOPS if esize == 8 else FP32_PEAK_TFLOPS
    hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "alg_bytes_per_launch": bpl, "alg_bytes_per_cell": alg_bytes_per_cell(NCELL, esize),
           "alg_bytes_per_cell_reading": "g = 3 guard layers from one neighbour slice (s = 1)",
           "alg_bytes_per_cell_radius2": alg_bytes_radius2(NCELL, esize), "peak_kind": peak_kind}
    alu = {"bound": "alu", "achieved": tfs, "peak": fpeak, "unit": "TFLOP/s", "frac": tfs / fpeak,
           "alg_flops_per_launch": fpl, "alg_flops_per_cell": flops_per_cell,
           "peak_kind": "derived: 152 SMs x %s x 2.07 GHz" % ("2 FP64 FMA/cycle" if esize == 8 else "128 FP32 lanes")}
    if esize == 8:
        return dict(alu, hbm=hbm)
    return dict(hbm, alu=alu)


def run_form(lay, state_dev, precision, steps, warmup, td, variant=-1, riemann=0, nonideal=None):
    """Time `steps` global steps of one precision form (HLL or HLLD face
    fluxes, optionally with the non-ideal terms) from the initial state."""
    import torch
    from paper_1705_10774_gb300.dispatch import Dispatch
    stream = torch.cuda.current_stream()
    g = Dispatch(lay.n, lay.lo, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                 precision=precision, time_mode=0, timing=1, variant=variant, riemann=riemann,
                 stream=stream.cuda_stream, **(nonideal or {}))
    g.set_state(*state_dev)
    if variant < 0:
        g.tuned = g.autotune(reps=2)      # pick the fastest compiled variant (untimed set-up)
    else:
        g.tuned = (variant, {})
    if warmup:
        g.advance(max_sweeps=warmup)
    g.set_state(*state_dev)
    torch.cuda.synchronize()
    if td is not None:
        td.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = g.advance(max_sweeps=steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if td is not None:
        td.barrier()
    ms = e0.elapsed_time(e1)
    return g, st, ms


def traffic_of(variant, ncells):
    per = TRAFFIC_PER_CELL.get(variant)
    return None if per is None else per * ncells


def side_forms(args, td, peak, peak_kind):
    """The side forms on the 256^3 turbulence input: FP64 with FMA and
    without (bit-identical to the oracle), FP32, HLLD faces and the non-ideal
    terms in both precisions."""
    import torch
    lay, state = make_side_input()
    state_dev = [torch.from_numpy(a).cuda() for a in state]
    ncells = int(np.prod(lay.base_cells))
    forms = {}
    runs = [("f64", F64_PRECISION, 0, None), ("f64_exact", 0, 0, None), ("f32", 1, 0, None)]
    if not args.no_hlld:
        runs += [("f64_hlld", F64_PRECISION, 1, None), ("f32_hlld", 1, 1, None)]
    if not args.no_nonideal:
        runs += [("f64_nonideal", F64_PRECISION, 0, NONIDEAL), ("f32_nonideal", 1, 0, NONIDEAL)]
    for name, prec, rs, ni in runs:
        if prec == 1 and args.no_f32:
            continue
        sd = [a.float() for a in state_dev] if prec == 1 else state_dev
        g, st, ms = run_form(lay, sd, prec, args.steps, args.warmup, td, riemann=rs, nonideal=ni)
        ms = max_over_ranks(td, ms)
        k = st["kernel_ms"] / max(st["kernel_launches"], 1)
        r = {"value": sum_over_ranks(td, float(st["cell_updates"])) / (ms * 1e-3), "ms_per_step": ms / args.steps,
             "dtype": "f32" if prec == 1 else "f64", "kernel": "update_kernel variant %d" % g.tuned[0],
             "kernel_ms_avg": k}
        if ni is None:
            r["roofline"] = rooflines(ncells, 4 if prec == 1 else 8, k, peak, peak_kind,
                                      ALG_FLOPS_PER_CELL_HLLD if rs else ALG_FLOPS_PER_CELL)
            r["roofline"]["traffic"] = traffic_of(g.tuned[0], ncells)
        if name == "f64_exact":
            r["note"] = "no FMA contraction; bit-identical to the FP64 oracle"
        elif rs:
            r["note"] = "HLLD face fluxes (Miyoshi & Kusano 2005)"
        elif ni:
            r["note"] = "Ohmic and ambipolar EMFs and their Poynting flux, %s" % NONIDEAL
        forms[name] = r
        g.close()
        del sd
    return {"workload": SIDE_WORKLOAD, "forms": forms}


def gpu_arm(args):
    import torch
    td, rank, ws = dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1705_10774_gb300 import dispatch as D
    D.load()
    peak, peak_kind = measured_peaks()

    if args.form != "both":
        # profiling runs: one form on the 256^3 turbulence input (or --patches)
        lay, state = make_side_input(args.patches or SIDE_PATCHES)
        state_dev = [torch.from_numpy(a).cuda() for a in state]
        prec = {"f32": 1, "f64": F64_PRECISION, "f64_exact": 0}[args.form]
        sd = [a.float() for a in state_dev] if prec else state_dev
        g, st, ms = run_form(lay, sd, prec, args.steps, args.warmup, td, args.variant, args.riemann,
                             NONIDEAL if args.nonideal else None)
        if rank == 0:
            print(json.dumps({"form": args.form, "riemann": args.riemann, "variant": g.tuned[0],
                              "patches": lay.npatch, "ms_per_step": ms / args.steps,
                              "kernel_ms_avg": st["kernel_ms"] / max(st["kernel_launches"], 1),
                              "cell_updates_per_s": st["cell_updates"] / (ms * 1e-3)}))
        return

    P = args.patches or PATCHES
    lay, state = make_input(P)
    ncells = int(np.prod(lay.base_cells))
    state_dev = [torch.from_numpy(a).cuda() for a in state]
    with Clocks(local) as clk:
        g, st, ms = run_form(lay, state_dev, F64_PRECISION, args.steps, args.warmup, td)
    ms_max = max_over_ranks(td, ms)
    cells_all = sum_over_ranks(td, float(st["cell_updates"]))
    value = cells_all / (ms_max * 1e-3)
    kavg = st["kernel_ms"] / max(st["kernel_launches"], 1)
    roof = rooflines(ncells, 8, kavg, peak, peak_kind)
    roof.update({"traffic": traffic_of(g.tuned[0], ncells), "kernel": "update_kernel variant %d" % g.tuned[0],
                 "kernel_ms_avg": kavg, "autotune_ms_per_variant": g.tuned[1]})
    launches = int(st["kernel_launches"] + st["plan_launches"])
    g.close()

    forms = {"f64": {"value": value, "ms_per_step": ms_max / args.steps, "dtype": "f64"}}
    v32 = None
    if not args.no_f32:
        state32 = [a.float() for a in state_dev]
        del state_dev
        torch.cuda.empty_cache()
        g32, st32, ms32 = run_form(lay, state32, 1, args.steps, args.warmup, td)
        ms32_max = max_over_ranks(td, ms32)
        v32 = sum_over_ranks(td, float(st32["cell_updates"])) / (ms32_max * 1e-3)
        k32 = st32["kernel_ms"] / max(st32["kernel_launches"], 1)
        r32 = rooflines(ncells, 4, k32, peak, peak_kind)
        r32.update({"traffic": traffic_of(g32.tuned[0], ncells), "kernel": "update_kernel variant %d" % g32.tuned[0],
                    "kernel_ms_avg": k32, "autotune_ms_per_variant": g32.tuned[1]})
        forms["f32"] = {"value": v32, "ms_per_step": ms32_max / args.steps, "dtype": "f32", "roofline": r32}
        g32.close()
        del state32
    else:
        del state_dev
    torch.cuda.empty_cache()

    side = None if args.no_side else side_forms(args, td, peak, peak_kind)
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        e2e = e2e_measure(lay, state, min(args.steps, args.e2e_steps), td)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lay, state)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "value_f32": v32, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(P), "patches": lay.npatch, "cells_per_patch": [NCELL] * 3,
                       "cells": ncells, "time_mode": "global", "precision": "f64 (fused multiply-adds)",
                       "l2": "inputs larger than L2 (%.1f GB per FP64 slice)" % (sum(a.nbytes for a in state) / 1e9),
                       "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "roofline": roof,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "forms": forms,
            "side": side,
        }
        print(json.dumps(out))
    if td is not None:
        td.barrier()
        td.destroy_process_group()


def e2e_measure(lay, state, steps, td):
    """Through the library's own host-buffer path: every step loads the input
    from pinned host memory with dsp_set_state(on_device = 0) -- the library
    copies it into its device staging buffer and scatters it into the
    slices --, advances one global step, and reads the new state back into
    pinned host memory with dsp_get_state(on_device = 0) (gather kernel,
    then the library's copy to the host).  Each call synchronises, so the
    copies are in line with the sweeps."""
    import torch
    from paper_1705_10774_gb300.dispatch import Dispatch
    pinned = [torch.from_numpy(a).pin_memory() for a in state]
    outs = [torch.empty_like(a).pin_memory() for a in pinned]
    stream = torch.cuda.current_stream()
    g = Dispatch(lay.n, lay.lo, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                 precision=F64_PRECISION, time_mode=0, stream=stream.cuda_stream)
    h_in = sum(a.numel() * a.element_size() for a in pinned)
    h_out = sum(a.numel() * a.element_size() for a in outs)
    g.set_state(*pinned)                    # allocates the library's staging buffer before timing
    g.autotune(reps=2)
    g.set_state(*pinned)
    g.advance(max_sweeps=1)
    g.get_state(out=outs)
    torch.cuda.synchronize()
    if td is not None:
        td.barrier()
    cells = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        g.set_state(*pinned)
        st = g.advance(max_sweeps=1)
        g.get_state(out=outs)
        cells += st["cell_updates"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(td, dt)
    cells = sum_over_ranks(td, cells)
    g.close()
    del pinned, outs
    return {"value": cells / dt, "unit": UNIT, "h2d_bytes_per_step": h_in, "d2h_bytes_per_step": h_out,
            "steps": steps,
            "path": "dsp_set_state / dsp_advance(1 sweep) / dsp_get_state with pinned host pointers "
                    "(on_device = 0): the library's own copies through its device staging buffer"}


def oracle_sample(lay, state, steps, warmup, per_step=32):
    """The FP64 oracle as it stands on a bounded sample of the workload: each
    step updates `per_step` patches (a fixed seeded permutation) from the
    initial state with the global step, spread over the host cores (the
    oracle's update releases the interpreter lock).  Returns (cell-updates/s,
    seconds, cores, patch updates)."""
    from oracle import Oracle
    o = Oracle(lay.n, lay.lo, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    o.set_state(*state)
    dt = min(o.patch_dt(i) for i in range(lay.npatch))
    cores = os.cpu_count() or 1
    order = np.random.default_rng(1).permutation(lay.npatch)
    pool = ThreadPoolExecutor(max_workers=cores)

    def step(k):
        ids = [int(order[(k * per_step + j) % lay.npatch]) for j in range(per_step)]
        list(pool.map(lambda i: o.update_patch(i, dt), ids))

    for k in range(warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(steps):
        step(warmup + k)
    el = time.perf_counter() - t0
    pool.shutdown()
    cells = steps * per_step * NCELL ** 3
    # one core: the same updates one after another
    t1 = time.perf_counter()
    for j in range(4):
        o.update_patch(int(order[j]), dt)
    d1 = time.perf_counter() - t1
    return cells / el, el, cores, steps * per_step, 4 * NCELL ** 3 / d1


def cpu_baseline(lay, state, steps=16):
    v, el, cores, nup, v1 = oracle_sample(lay, state, steps, 1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d patch updates of 32^3 from the %d^3 input with its global step, over %d threads "
                      "(%.1f s)" % (nup, lay.base_cells[0], cores, el),
            "single_core": {"value": v1, "unit": UNIT, "cores": 1, "sample": "4 patch updates of 32^3 in sequence"}}


def reference_arm(args):
    """The FP64 CPU oracle, timed on the host cores; each step is a bounded
    sample of the workload: 32 patch updates (1.05M cell-updates) of the
    benchmark's input with its global step, spread over the cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    P = args.patches or PATCHES
    lay, state = make_input(P)
    value, el, cores, nup, _ = oracle_sample(lay, state, args.steps, args.warmup)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(P), "patches": lay.npatch, "cells_per_patch": [NCELL] * 3,
                   "sample_per_step": "32 patch updates"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "32 patch updates of 32^3 per step, %d steps" % args.steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def lts_arm(args):
    """Local time steps on the 4096-patch input (16^3 patches of 16^3 cells,
    log-normal density, hot sphere): both dispatchers, FP64 (FMA) and FP32,
    to t_end; and the same input with one global step per sweep, for the
    ratio of cell-updates needed (the paper's local-time-step advantage)."""
    import torch
    from paper_1705_10774_gb300 import ics
    from paper_1705_10774_gb300.dispatch import Dispatch
    lay, f = ics.config_lts(patches=16, n=16)
    state = [torch.from_numpy(a).cuda() for a in ics.to_patches(lay, f)]
    stream = torch.cuda.current_stream()
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, stream=stream.cuda_stream)
    out = {"workload": "local steps, 4096 patches of 16^3 (256^3), log-normal rho, hot sphere", "t_end": args.t_end}
    for name, prec, disp, mode in [("f64_queue", F64_PRECISION, 0, 1), ("f64_sweep_graph", F64_PRECISION, 1, 1),
                                   ("f32_queue", 1, 0, 1), ("f32_sweep_graph", 1, 1, 1), ("f32_global", 1, 1, 0)]:
        st_in = [a.float() for a in state] if prec == 1 else state
        g = Dispatch(lay.n, lay.lo, precision=prec, dispatcher=disp, time_mode=mode, graph=1, timing=1,
                     sched_capacity=1 << 24 if mode == 1 and disp == 1 else 0, **kw)
        g.set_state(*st_in)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = g.advance(t_end=args.t_end)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r = {"ms": ms, "cell_updates": st["cell_updates"], "patch_updates": st["patch_updates"],
             "sweeps": st["sweeps"], "cell_updates_per_s": st["cell_updates"] / (ms * 1e-3),
             "pressure_floor_cells": st["floors"], "first_order_fallback_cells": st["fallbacks"]}
        if name == "f64_sweep_graph" or name == "f32_sweep_graph":
            _, _, dts = g.schedule()
            lv, cnt = np.unique(dts, return_counts=True)
            r["dt_levels"] = int(len(lv))
            r["dt_ratio_max_min"] = float(lv.max() / lv.min())
            # patch updates per step size (the clipped last steps to t_end included)
            r["updates_per_dt"] = {"%.6e" % a: int(b) for a, b in zip(lv, cnt)}
        out[name] = r
        g.close()
    out["lts_over_global_cell_updates"] = out["f32_queue"]["cell_updates"] / out["f32_global"]["cell_updates"]
    print(json.dumps(out))


def kitp_arm(args):
    """Sec. 5.1's decaying-turbulence check on the benchmark's 256^3 input
    (which stands in for the KITP snapshot): one patch of 256^3 against 512
    patches of 32^3 with local steps, and the 512-patch run at another
    Courant number, FP32, to t_end (default 0.2).  Reports the
    root-mean-square velocity of each run, their relative differences, and
    the cell-updates each needed (the local-time-step saving)."""
    import torch
    from paper_1705_10774_gb300 import ics
    from paper_1705_10774_gb300.dispatch import Dispatch
    lay512, f = ics.config_turbulence(seed=10774, patches=SIDE_PATCHES, n=NCELL, mach=2.0)
    lay1 = ics.cartesian(1, SIDE_PATCHES * NCELL)
    t_end = args.t_end if args.t_end != 0.01 else 0.2
    runs = {}
    for name, lay, cfl in (("1_patch", lay1, 0.4), ("512_patches", lay512, 0.4), ("512_patches_cfl0.3", lay512, 0.3)):
        st = [torch.from_numpy(a).float().cuda() for a in ics.to_patches(lay, f)]
        g = Dispatch(lay.n, lay.lo, gamma=f.gamma, cfl=cfl, base_cells=lay.base_cells, box_len=lay.box_len,
                     time_mode=1, precision=1, graph=1)
        g.set_state(*st)
        del st
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = g.advance(t_end=t_end)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        U = g.get_state()[0]
        g.close()
        npch = lay.npatch
        U = U.reshape(npch, 5, -1)
        rho = U[:, 0].astype(np.float64)
        v2 = (U[:, 1].astype(np.float64) ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / rho ** 2
        runs[name] = {"cfl": cfl, "v_rms": float(np.sqrt(v2.mean())), "cell_updates": res["cell_updates"],
                      "sweeps": res["sweeps"], "seconds": el, "cell_updates_per_s": res["cell_updates"] / el,
                      "rho_sorted": np.sort(rho.ravel())}
    r1, r5, r3 = runs["1_patch"], runs["512_patches"], runs["512_patches_cfl0.3"]
    out = {"workload": "decaying MHD turbulence 256^3 (Mach 2, beta 1), FP32, local steps, t = 0 to %g" % t_end,
           "v_rms_rel_diff_1_vs_512_patches": abs(r5["v_rms"] - r1["v_rms"]) / r1["v_rms"],
           "v_rms_rel_diff_cfl_0.4_vs_0.3": abs(r5["v_rms"] - r3["v_rms"]) / r5["v_rms"],
           "cell_updates_512_over_1_patch": r5["cell_updates"] / r1["cell_updates"],
           # the density distributions (cell order differs between layouts)
           "density_quantile_rel_diff_1_vs_512": float(np.max(np.abs(r5["rho_sorted"] - r1["rho_sorted"]))
                                                       / np.max(r1["rho_sorted"])),
           "runs": {k: {q: v for q, v in r.items() if q != "rho_sorted"} for k, r in runs.items()}}
    print(json.dumps(out))


def grace_arm(args):
    """Eq. 1's grace and the order of the time inter- and extrapolation of
    guard values (Sec. 3 B) on the local-step input (4096 patches of 16^3),
    FP64 with FMA, sweeps replayed from CUDA graphs, to t_end: sweeps,
    updates, time and the state's relative L1 distance from g = 0 with
    linear interpolation."""
    import torch
    from paper_1705_10774_gb300 import ics
    from paper_1705_10774_gb300.dispatch import Dispatch
    lay, f = ics.config_lts(patches=16, n=16)
    state = [torch.from_numpy(a).cuda() for a in ics.to_patches(lay, f)]
    stream = torch.cuda.current_stream()
    kw = dict(gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, stream=stream.cuda_stream,
              precision=F64_PRECISION, dispatcher=1, time_mode=1, graph=1)
    out = {"workload": "local steps, 4096 patches of 16^3 (256^3), log-normal rho, hot sphere", "t_end": args.t_end,
           "runs": []}
    ref = None
    for grace, order, ns in ((0.0, 1, 3), (0.05, 1, 3), (0.3, 1, 3), (0.6, 1, 3), (0.0, 2, 3), (0.6, 2, 4)):
        g = Dispatch(lay.n, lay.lo, grace=grace, time_order=order, nslices=ns, **kw)
        g.set_state(*state)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = g.advance(t_end=args.t_end)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s1 = g.get_state()
        if ref is None:
            ref = s1
        num = sum(float(np.abs(a - b).sum()) for a, b in zip(s1, ref))
        den = sum(float(np.abs(b).sum()) for b in ref)
        out["runs"].append({"grace": grace, "time_order": order, "nslices": ns, "sweeps": st["sweeps"],
                            "patch_updates": st["patch_updates"], "ms": ms,
                            "cell_updates_per_s": st["cell_updates"] / (ms * 1e-3), "relative_L1_vs_first": num / den})
        g.close()
    print(json.dumps(out))


def orszag_tang_arm(args):
    """3-D Orszag-Tang vortex: FP32 state against FP64 on the same GPU, from
    the same input to the same time: relative L1 of density, momentum,
    energy and field, conservation drift, max div B (per max |B|)."""
    import torch
    from paper_1705_10774_gb300 import ics
    from paper_1705_10774_gb300.dispatch import Dispatch
    lay, state = ics.orszag_tang_patches(patches=args.patches or PATCHES, n=NCELL)
    stream = torch.cuda.current_stream()
    kw = dict(gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=0,
              graph=1, stream=stream.cuda_stream)
    res = {}
    for name, prec in (("f64", F64_PRECISION), ("f32", 1)):
        g = Dispatch(lay.n, lay.lo, precision=prec, **kw)
        g.set_state(*state)
        d0 = g.diagnostics()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.advance(t_end=args.t_end)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        d1 = g.diagnostics()
        res[name] = dict(state=g.get_state(), d0=d0, d1=d1, st=st, s=el)
        g.close()
    a, b = res["f64"]["state"], res["f32"]["state"]
    npch = lay.npatch
    A, B = a[0].reshape(npch, 5, -1), b[0].reshape(npch, 5, -1)
    l1 = lambda x, y: float(np.sum(np.abs(x - y)) / np.sum(np.abs(x)))
    errs = {"rho": l1(A[:, 0], B[:, 0]), "m_x": l1(A[:, 1], B[:, 1]), "m_y": l1(A[:, 2], B[:, 2]),
            "m_z": l1(A[:, 3], B[:, 3]), "E": l1(A[:, 4], B[:, 4]), "b_x": l1(a[1], b[1]), "b_y": l1(a[2], b[2]),
            "b_z": l1(a[3], b[3]), "mom": l1(A[:, 1:4], B[:, 1:4]), "b": l1(np.concatenate(a[1:]), np.concatenate(b[1:]))}
    drift = {}
    for name in ("f64", "f32"):
        d0, d1 = res[name]["d0"], res[name]["d1"]
        drift[name] = {"mass": abs(d1["mass"] - d0["mass"]) / abs(d0["mass"]),
                       "energy": abs(d1["energy"] - d0["energy"]) / abs(d0["energy"]),
                       "max_divb_over_max_b": d1["max_divb"] / d1["max_b"],
                       "steps": res[name]["st"]["sweeps"], "seconds": res[name]["s"],
                       "cell_updates_per_s": res[name]["st"]["cell_updates"] / res[name]["s"]}
    print(json.dumps({"workload": "Orszag-Tang %d^3 (%d patches of %d^3)" % (lay.base_cells[0], npch, NCELL),
                      "t_end": args.t_end, "f32_vs_f64_relative_L1": errs, "per_form": drift}))


def mixed_arm(args):
    """Mixed patch sizes on one level (the coarse level of the uneven batched
    solve): 512^3 cut into 96^3 super-blocks of 16^3, 24^3 or 32^3 patches
    (seeded, ~40/30/30 % by count) plus 32^3 remainder slabs; turbulence input
    as the benchmark's (Mach 2, beta 1); FP32 state, local steps, sweeps
    replayed from CUDA graphs."""
    import torch
    from paper_1705_10774_gb300 import ics
    from paper_1705_10774_gb300.dispatch import Dispatch
    lay = ics.mixed_blocks(args.blocks, 96, remainder=32, seed=17)
    X, Y, Z = lay.base_cells
    rng = np.random.default_rng(10774)
    v = ics.solenoidal_velocity((Z, Y, X), lay.box_len, 1.0, 4.0, 2.0, rng)
    f = ics.Fields(rho=np.ones((Z, Y, X)), v=v, p=np.full((Z, Y, X), 0.6), bx=np.full((Z, Y, X), np.sqrt(1.2)),
                   by=np.zeros((Z, Y, X)), bz=np.zeros((Z, Y, X)), gamma=5.0 / 3.0)
    state = [torch.from_numpy(a.astype(np.float32)).cuda() for a in ics.to_patches(lay, f)]
    del f, v
    stream = torch.cuda.current_stream()
    g = Dispatch(lay.n, lay.lo, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                 precision=1, time_mode=1, graph=1, timing=1, stream=stream.cuda_stream,
                 dispatcher=args.dispatcher)
    g.set_state(*state)
    if not args.no_tune:
        g.autotune(reps=2)                    # a variant and z run per patch size
    g.set_state(*state)
    g.advance(t_end=args.t_end / 4)           # warm-up
    g.set_state(*state)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = g.advance(t_end=args.t_end)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sizes, counts = np.unique(lay.n[:, 0], return_counts=True)
    print(json.dumps({"workload": "mixed 16/24/32 patches, %d^3, %d patches" % (X, lay.npatch),
                      "dispatcher": "ready queue" if args.dispatcher == 0 else "sweeps from CUDA graphs",
                      "patch_sizes": dict(zip(map(int, sizes), map(int, counts))), "t_end": args.t_end,
                      "ms": ms, "cell_updates": st["cell_updates"], "sweeps": st["sweeps"],
                      "cell_updates_per_s": st["cell_updates"] / (ms * 1e-3), "tuning": g.tuning(),
                      "tuning_candidates": getattr(g, "tuning_log", [])}))
    g.close()


def amr_arm(args):
    """Two refinement levels with mixed patch sizes (the uneven batched solve
    of Sec. 5.2 stood in for by synthetic data): level 0 = 512^3 over the box
    in 96^3 super-blocks of 16^3 / 24^3 / 32^3 patches plus 32^3 remainder
    slabs; level 1 = 256^3 cells at dx/2 over [3/8, 5/8]^3, tiled the same
    way (remainder 64 cells in 32^3 patches).  The benchmark's turbulence
    input on level 0 (rms |v| = 2, beta = 1); level-1 cells take their
    level-0 parent's velocity.  FP32 state, local steps, sweeps replayed from
    CUDA graphs, autotuned."""
    import torch
    from paper_1705_10774_gb300 import ics
    from paper_1705_10774_gb300.dispatch import Dispatch
    lay, arrays = ics.config_two_level(args.blocks)
    state = [torch.from_numpy(a).cuda() for a in arrays]
    del arrays
    stream = torch.cuda.current_stream()
    g = Dispatch(lay.n, lay.lo, level=lay.levels, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells,
                 box_len=lay.box_len, precision=1, time_mode=1, graph=1, timing=1, stream=stream.cuda_stream,
                 sched_capacity=1 << 22)
    g.set_state(*state)
    tuned = g.autotune(reps=2) if not args.no_tune else (-1, {})
    g.set_state(*state)
    g.advance(t_end=args.t_end / 4)           # warm-up
    g.set_state(*state)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = g.advance(t_end=args.t_end)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    p, _, dts = g.schedule()
    lev = lay.levels[p]
    cells = np.prod(lay.n, axis=1)[p]
    out = {"workload": "two levels: 512^3 level 0 + 256^3 level 1 over [3/8,5/8]^3, mixed 16/24/32 patches",
           "patches": int(lay.npatch), "patches_per_level": [int((lay.levels == l).sum()) for l in (0, 1)],
           "cells": int(np.prod(lay.n, axis=1).sum()), "t_end": args.t_end, "ms": ms,
           "cell_updates": st["cell_updates"], "sweeps": st["sweeps"],
           "cell_updates_per_level": [int(cells[lev == l].sum()) for l in (0, 1)],
           "dt_per_level": [sorted(set(np.unique(dts[lev == l]).tolist()))[:4] for l in (0, 1)],
           "cell_updates_per_s": st["cell_updates"] / (ms * 1e-3), "variant": tuned[0],
           "tuning": g.tuning(), "tuning_candidates": getattr(g, "tuning_log", []),
           "kernel_ms": st["kernel_ms"]}
    print(json.dumps(out))
    g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-f32", action="store_true")
    ap.add_argument("--form", default="both", choices=["both", "f64", "f64_exact", "f32"],
                    help="f64 / f32: time only that form and print a short line (profiling runs)")
    ap.add_argument("--patches", type=int, default=0,
                    help="patches per axis of 32^3 (default: 16 for the benchmark line, 8 for --form runs)")
    ap.add_argument("--no-side", action="store_true", help="skip the 256^3 side forms")
    ap.add_argument("--variant", type=int, default=-1,
                    help="--form runs: use this compiled kernel variant instead of autotuning")
    ap.add_argument("--riemann", type=int, default=0, choices=[0, 1],
                    help="--form runs: face fluxes, 0 = HLL, 1 = HLLD")
    ap.add_argument("--no-hlld", action="store_true", help="skip the HLLD forms of the benchmark line")
    ap.add_argument("--no-nonideal", action="store_true", help="skip the non-ideal forms of the benchmark line")
    ap.add_argument("--nonideal", action="store_true",
                    help="--form runs: with the non-ideal terms of the benchmark's non-ideal forms")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="turbulence",
                    choices=["turbulence", "lts", "orszag-tang", "mixed", "amr", "grace", "kitp"],
                    help="lts / orszag-tang: side measurements (one JSON line each), not the benchmark line")
    ap.add_argument("--t-end", type=float, default=0.01, help="end time of the lts / orszag-tang / mixed runs")
    ap.add_argument("--blocks", type=int, default=5, help="96^3 super-blocks per axis of the mixed run")
    ap.add_argument("--no-tune", action="store_true", help="mixed / amr runs: keep the default variant")
    ap.add_argument("--dispatcher", type=int, default=1, choices=[0, 1],
                    help="mixed run: 1 sweeps replayed from CUDA graphs, 0 the persistent ready queue")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "lts":
        return lts_arm(args)
    if args.workload == "orszag-tang":
        return orszag_tang_arm(args)
    if args.workload == "mixed":
        return mixed_arm(args)
    if args.workload == "amr":
        return amr_arm(args)
    if args.workload == "grace":
        return grace_arm(args)
    if args.workload == "kitp":
        return kitp_arm(args)
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
