#!/usr/bin/env python
"""Benchmark of the per-patch update: MHD cell-updates/s on one GB300.

Workload (one line per run): decaying MHD turbulence on a periodic 256^3 box
cut into 8^3 = 512 patches of 32^3 cells, FP64, one global power-of-two
Courant step per sweep (C = 0.4), seeded solenoidal Mach-2 velocity with
E(k) ~ k^-2 on 1 <= |k|/2pi <= 4, uniform B along x at beta = 1.  A bench
"step" is one sweep: every patch fills its guard zones, advances one step and
publishes it.  The state (1.07 GB per slice in FP64) is larger than L2, so no
flush is needed between steps.  The FP32-state form of the same run, both
forms with HLLD face fluxes and both with the non-ideal Ohmic and ambipolar
terms are measured too and reported under "forms".

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (32 patch updates per step).
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
PATCHES, NCELL = 8, 32
WORKLOAD = "decaying MHD turbulence, 256^3 periodic, 512 patches of 32^3, global dt, CFL 0.4"
HBM_FALLBACK_GBS = 6800.0
# the timed FP64 form: FP64 state and arithmetic with fused multiply-adds
# (checked against the FP64 oracle to 1e-11); the FMA-free build that matches
# the oracle bit for bit is timed too and reported as forms.f64_exact
F64_PRECISION = 2
# coefficients of the non-ideal forms: Ohmic resistivity, and the C-shock
# experiment's ambipolar drift coefficient and ion density (Sec. 5.4)
NONIDEAL = dict(eta=1e-4, gamma_ad=75.0, rho_i=1.0)

# DRAM bytes (read + write) per update-kernel launch of the full workload,
# by compiled variant, from ncu's dram__bytes_read.sum + dram__bytes_write.sum
# (FP64: a 216-patch capture of the same kernel, scaled by cells; FP32: the
# full workload); a variant without an entry reports null.
TRAFFIC_F64 = {2: (550.772736e6 + 421.459712e6) * 512 / 216, 3: (551.252736e6 + 421.417472e6) * 512 / 216,
               4: (552.264960e6 + 424.443648e6) * 512 / 216}
TRAFFIC_F32 = {5: 626.309120e6 + 509.839360e6}
# the same for the HLLD variants (FP64 FMA: the 216-patch capture, scaled)
TRAFFIC_F64_HLLD = {10: (538.658560e6 + 421.405696e6) * 512 / 216}
TRAFFIC_F32_HLLD = {11: 622.772736e6 + 510.983424e6}


def radius2_guard_fraction(n):
    return ((n + 4) ** 3 - n ** 3) / n ** 3


def alg_bytes_per_cell(n, esize, sbar=1.0):
    """Algorithmic HBM bytes per cell-update: read and write the 8 stored
    fields once, plus the guard shell the stencil reads (radius 2), taken
    from sbar neighbour slices."""
    V = 8
    return esize * (2 * V + sbar * radius2_guard_fraction(n) * V)


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
    from paper_1705_10774_gb300 import ics
    lay, f = ics.config_turbulence(seed=10774, patches=patches, n=NCELL, mach=2.0)
    return lay, f, ics.to_patches(lay, f)


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
           "alg_bytes_per_launch": bpl, "peak_kind": peak_kind}
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


def gpu_arm(args):
    import torch
    td, rank, ws = dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1705_10774_gb300 import dispatch as D
    D.load()
    lay, f, state = make_input(args.patches if args.form != "both" else PATCHES)
    state_dev = [torch.from_numpy(a).cuda() for a in state]
    ncells = int(np.prod(lay.base_cells))
    peak, peak_kind = measured_peaks()

    if args.form != "both":
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
    with Clocks(local) as clk:
        g, st, ms = run_form(lay, state_dev, F64_PRECISION, args.steps, args.warmup, td)
    ms_max = max_over_ranks(td, ms)
    cells_all = sum_over_ranks(td, float(st["cell_updates"]))
    value = cells_all / (ms_max * 1e-3)
    kavg = st["kernel_ms"] / max(st["kernel_launches"], 1)
    roof = rooflines(ncells, 8, kavg, peak, peak_kind)
    roof.update({"traffic": TRAFFIC_F64.get(g.tuned[0]), "kernel": "update_kernel variant %d" % g.tuned[0],
                 "kernel_ms_avg": kavg,
                 "autotune_ms_per_variant": g.tuned[1]})
    g.close()

    forms = {}
    if args.form == "both":
        ge, ste, mse = run_form(lay, state_dev, 0, args.steps, args.warmup, td)
        mse = max_over_ranks(td, mse)
        forms["f64_exact"] = {"value": sum_over_ranks(td, float(ste["cell_updates"])) / (mse * 1e-3),
                              "ms_per_step": mse / args.steps, "dtype": "f64",
                              "kernel_ms_avg": ste["kernel_ms"] / max(ste["kernel_launches"], 1),
                              "note": "no FMA contraction; bit-identical to the FP64 oracle"}
        ge.close()

    if not args.no_f32 and args.form == "both":
        state32 = [a.float() for a in state_dev]
        g32, st32, ms32 = run_form(lay, state32, 1, args.steps, args.warmup, td)
        ms32_max = max_over_ranks(td, ms32)
        v32 = sum_over_ranks(td, float(st32["cell_updates"])) / (ms32_max * 1e-3)
        k32 = st32["kernel_ms"] / max(st32["kernel_launches"], 1)
        r32 = rooflines(ncells, 4, k32, peak, peak_kind)
        r32.update({"traffic": TRAFFIC_F32.get(g32.tuned[0]), "kernel": "update_kernel variant %d" % g32.tuned[0],
                    "kernel_ms_avg": k32, "autotune_ms_per_variant": g32.tuned[1]})
        forms["f32"] = {"value": v32, "ms_per_step": ms32_max / args.steps, "dtype": "f32", "roofline": r32}
        g32.close()
        del state32

    if not args.no_hlld and args.form == "both":
        # the same run with HLLD face fluxes (edge EMFs stay upwind HLL)
        for name, prec in (("f64_hlld", F64_PRECISION), ("f32_hlld", 1)):
            if prec == 1 and args.no_f32:
                continue
            sd = [a.float() for a in state_dev] if prec == 1 else state_dev
            gh, sth, msh = run_form(lay, sd, prec, args.steps, args.warmup, td, riemann=1)
            msh = max_over_ranks(td, msh)
            kh = sth["kernel_ms"] / max(sth["kernel_launches"], 1)
            rh = rooflines(ncells, 4 if prec == 1 else 8, kh, peak, peak_kind, ALG_FLOPS_PER_CELL_HLLD)
            rh.update({"traffic": (TRAFFIC_F32_HLLD if prec == 1 else TRAFFIC_F64_HLLD).get(gh.tuned[0]),
                       "kernel": "update_kernel variant %d" % gh.tuned[0], "kernel_ms_avg": kh})
            forms[name] = {"value": sum_over_ranks(td, float(sth["cell_updates"])) / (msh * 1e-3),
                           "ms_per_step": msh / args.steps, "dtype": "f32" if prec == 1 else "f64",
                           "roofline": rh, "note": "HLLD face fluxes (Miyoshi & Kusano 2005)"}
            gh.close()
            del sd

    if not args.no_nonideal and args.form == "both":
        # the same run with the non-ideal Ohmic and ambipolar terms (Sec. 4.3)
        for name, prec in (("f64_nonideal", F64_PRECISION), ("f32_nonideal", 1)):
            if prec == 1 and args.no_f32:
                continue
            sd = [a.float() for a in state_dev] if prec == 1 else state_dev
            gn, stn, msn = run_form(lay, sd, prec, args.steps, args.warmup, td, nonideal=NONIDEAL)
            msn = max_over_ranks(td, msn)
            forms[name] = {"value": sum_over_ranks(td, float(stn["cell_updates"])) / (msn * 1e-3),
                           "ms_per_step": msn / args.steps, "dtype": "f32" if prec == 1 else "f64",
                           "kernel": "update_kernel variant %d" % gn.tuned[0],
                           "kernel_ms_avg": stn["kernel_ms"] / max(stn["kernel_launches"], 1),
                           "note": "Ohmic and ambipolar EMFs and their Poynting flux, %s" % NONIDEAL}
            gn.close()
            del sd

    e2e = None
    if not args.no_e2e:
        e2e = e2e_measure(lay, state, min(args.steps, args.e2e_steps), td)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lay, state)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "patches": lay.npatch, "cells_per_patch": [NCELL] * 3,
                       "cells": ncells, "time_mode": "global", "precision": "f64",
                       "l2": "inputs larger than L2 (1.07 GB per slice)", "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "roofline": roof,
            "forms": {"f64": {"value": value, "ms_per_step": ms_max / args.steps}, **forms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(st["kernel_launches"] + st["plan_launches"]),
            "clocks": clk.summary(),
        }
        print(json.dumps(out))
    if td is not None:
        td.barrier()
        td.destroy_process_group()


def e2e_measure(lay, state, steps, td):
    """Through the public API with host buffers: every step copies the input
    state from pinned host memory to the device, loads it (dsp_set_state),
    advances one global step and reads the new state back into pinned host
    memory.  The copies run on a second CUDA stream into double-buffered
    device staging arrays, so that step k+1's input and step k-1's result
    cross the host link while step k's sweep runs; the loads, sweeps and
    reads stay on the context's stream in order."""
    import torch
    from paper_1705_10774_gb300.dispatch import Dispatch
    pinned = [torch.from_numpy(a).pin_memory() for a in state]
    outs = [[torch.empty_like(a).pin_memory() for a in pinned] for _ in range(2)]
    dev_in = [[torch.empty(a.shape, dtype=a.dtype, device="cuda") for a in pinned] for _ in range(2)]
    dev_out = [[torch.empty(a.shape, dtype=a.dtype, device="cuda") for a in pinned] for _ in range(2)]
    stream = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    g = Dispatch(lay.n, lay.lo, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                 precision=F64_PRECISION, time_mode=0, stream=stream.cuda_stream)
    h_in = sum(a.numel() * a.element_size() for a in pinned)
    h_out = sum(a.numel() * a.element_size() for a in outs[0])
    for buf in dev_in:
        for d, h in zip(buf, pinned):
            d.copy_(h)
    g.set_state(*dev_in[0])                         # allocate the library's buffers before timing
    g.autotune(reps=2)
    g.set_state(*[a.numpy() for a in pinned])
    g.advance(max_sweeps=1)
    g.get_state(out=dev_out[0])
    torch.cuda.synchronize()
    if td is not None:
        td.barrier()

    def h2d(k):
        with torch.cuda.stream(copy):
            for d, h in zip(dev_in[k % 2], pinned):
                d.copy_(h, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(copy)
        return ev

    cells = 0
    t0 = time.perf_counter()
    ev_in = {0: h2d(0)}
    ev_out = {}
    for k in range(steps):
        if k + 1 < steps:
            ev_in[k + 1] = h2d(k + 1)              # next input, while this step runs
        stream.wait_event(ev_in.pop(k))
        g.set_state(*dev_in[k % 2])
        st = g.advance(max_sweeps=1)
        if k - 2 in ev_out:                         # the staging array's previous read is done
            stream.wait_event(ev_out.pop(k - 2))
        g.get_state(out=dev_out[k % 2])
        done = torch.cuda.Event()
        done.record(stream)
        with torch.cuda.stream(copy):
            copy.wait_event(done)
            for h, d in zip(outs[k % 2], dev_out[k % 2]):
                h.copy_(d, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(copy)
            ev_out[k] = ev
        cells += st["cell_updates"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(td, dt)
    cells = sum_over_ranks(td, cells)
    g.close()
    return {"value": cells / dt, "unit": UNIT, "h2d_bytes_per_step": h_in, "d2h_bytes_per_step": h_out,
            "steps": steps, "copies": "pinned host <-> device on a second stream, overlapping the sweeps"}


def cpu_baseline(lay, state, target_s=12.0):
    """The FP64 oracle as it stands (OpenMP over the ready patches of a
    sweep), on the host cores: whole global steps of the same workload."""
    from oracle import Oracle
    o = Oracle(lay.n, lay.lo, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    o.set_state(*state)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    n = 0
    while True:
        o.advance(max_sweeps=1)
        n += 1
        if time.perf_counter() - t0 > target_s or n >= 8:
            break
    dt = time.perf_counter() - t0
    cells = o.stats()["cell_updates"]
    # one core: single patch updates (the oracle parallelises over patches only)
    step = min(o.patch_dt(i) for i in range(lay.npatch))
    t1 = time.perf_counter()
    for P in range(8):
        o.update_patch(P, step)
    d1 = time.perf_counter() - t1
    c1 = 8 * int(np.prod(lay.n[0]))
    return {"value": cells / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d global step(s) of the 256^3 / 512-patch workload (%d cell-updates, %.1f s)" % (n, cells, dt),
            "single_core": {"value": c1 / d1, "unit": UNIT, "cores": 1,
                            "sample": "8 patch updates of 32^3 (%d cell-updates, %.2f s)" % (c1, d1)}}


def reference_arm(args):
    """The FP64 CPU oracle, timed on the host cores; each step is a bounded
    sample of the workload: 32 patch updates (1.05M cell-updates) from the
    initial state, spread over the cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import Oracle
    lay, f, state = make_input()
    o = Oracle(lay.n, lay.lo, gamma=5.0 / 3.0, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len)
    o.set_state(*state)
    dt = min(o.patch_dt(i) for i in range(lay.npatch))
    cores = os.cpu_count() or 1
    per_step = 32
    order = np.random.default_rng(1).permutation(lay.npatch)
    pool = ThreadPoolExecutor(max_workers=cores)

    def step(k):
        ids = [int(order[(k * per_step + j) % lay.npatch]) for j in range(per_step)]
        list(pool.map(lambda i: o.update_patch(i, dt), ids))

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    el = time.perf_counter() - t0
    cells = args.steps * per_step * NCELL ** 3
    value = cells / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "patches": lay.npatch, "cells_per_patch": [NCELL] * 3,
                   "sample_per_step": "%d patch updates" % per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d patch updates of 32^3 per step, %d steps" % (per_step, args.steps)},
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
             "sweeps": st["sweeps"], "cell_updates_per_s": st["cell_updates"] / (ms * 1e-3)}
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
    lay512, f = ics.config_turbulence(seed=10774, patches=PATCHES, n=NCELL, mach=2.0)
    lay1 = ics.cartesian(1, PATCHES * NCELL)
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
    lay, f = ics.config_orszag_tang(patches=args.patches, n=NCELL)
    state = ics.to_patches(lay, f)
    del f
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
    errs = {"rho": l1(A[:, 0], B[:, 0]), "mom": l1(A[:, 1:4], B[:, 1:4]), "E": l1(A[:, 4], B[:, 4]),
            "b": l1(np.concatenate(a[1:]), np.concatenate(b[1:]))}
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


def cshock_arm(args):
    """Sec. 5.4's non-ideal C-shock experiments on the GPU (FP64 without
    FMA, bit-identical to the oracle): from the Table 1 discontinuity on a
    periodic box of 4 (300 cells, patches of 30 x 4 x 4; the shock at 3,
    far enough from the wrap), local steps and CUDA graphs, to t = 0.2
    (ambipolar) and 0.3 (Ohmic).  Reports the mean distance of B_y from the
    steady C-shock profile (the ODE of the conservation laws, aligned at the
    mid-value) over the jump, and the ratio of the largest to the smallest
    per-patch step."""
    import torch
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from cshock_ode import jump_input, most_common_steps, profile_error
    from paper_1705_10774_gb300 import ics
    from paper_1705_10774_gb300.dispatch import Dispatch
    out = {}
    for name, t_end in (("ad_iso", 0.2), ("ad_noniso", 0.2), ("ohm", 0.3)):
        lay, f, gamma, kw, xc = jump_input(name)
        g = Dispatch(lay.n, lay.lo, gamma=gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                     time_mode=1, graph=1, precision=0, sched_capacity=1 << 22, **kw)
        g.set_state(*ics.to_patches(lay, f))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.advance(t_end=t_end)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        By = ics.from_patches(lay, *g.get_state())[2][0, 0]
        steps = most_common_steps(g.schedule(), lay.npatch)
        out[name] = {"t_end": t_end, "profile_error": profile_error(name, xc, By, 3.0),
                     "step_ratio_between_patches": float(steps.max() / steps.min()),
                     "patch_updates": st["patch_updates"], "sweeps": st["sweeps"], "seconds": el,
                     "cell_updates_per_s": st["cell_updates"] / el, "coefficients": kw}
        g.close()
    print(json.dumps({"workload": "non-ideal C-shocks of Table 1, 300 cells over 4, 10 patches of 30x4x4",
                      "cases": out}))


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
                 precision=1, time_mode=1, graph=1, timing=1, stream=stream.cuda_stream)
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
                      "patch_sizes": dict(zip(map(int, sizes), map(int, counts))), "t_end": args.t_end,
                      "ms": ms, "cell_updates": st["cell_updates"], "sweeps": st["sweeps"],
                      "cell_updates_per_s": st["cell_updates"] / (ms * 1e-3)}))
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
    tuned = g.autotune(reps=2)
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
           "kernel_ms": st["kernel_ms"]}
    print(json.dumps(out))
    g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-f32", action="store_true")
    ap.add_argument("--form", default="both", choices=["both", "f64", "f64_exact", "f32"],
                    help="f64 / f32: time only that form and print a short line (profiling runs)")
    ap.add_argument("--patches", type=int, default=PATCHES,
                    help="patches per axis for --form runs (profiling on a smaller box)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="--form runs: use this compiled kernel variant instead of autotuning")
    ap.add_argument("--riemann", type=int, default=0, choices=[0, 1],
                    help="--form runs: face fluxes, 0 = HLL, 1 = HLLD")
    ap.add_argument("--no-hlld", action="store_true", help="skip the HLLD forms of the benchmark line")
    ap.add_argument("--no-nonideal", action="store_true", help="skip the non-ideal forms of the benchmark line")
    ap.add_argument("--nonideal", action="store_true",
                    help="--form runs: with the non-ideal terms of the benchmark's non-ideal forms")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="turbulence",
                    choices=["turbulence", "lts", "orszag-tang", "mixed", "amr", "cshock", "grace", "kitp"],
                    help="lts / orszag-tang: side measurements (one JSON line each), not the benchmark line")
    ap.add_argument("--t-end", type=float, default=0.01, help="end time of the lts / orszag-tang / mixed runs")
    ap.add_argument("--blocks", type=int, default=5, help="96^3 super-blocks per axis of the mixed run")
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
    if args.workload == "cshock":
        return cshock_arm(args)
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
