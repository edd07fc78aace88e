"""Build libdispatch_gpu.so in-tree with nvcc for sm_103a.

The FP64 translation units are compiled with -fmad=false (each product and
sum rounded on its own, as in the FP64 oracle); the FP32 update kernel keeps
fused multiply-adds.
"""
from __future__ import annotations

import os
import re
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libdispatch_gpu.so")
# the bounds-checked build: every global load and store of the update kernel
# is checked against the slice and guard buffers (DSP_ERR_BOUNDS, no trap)
OUT_DIR_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(OUT_DIR_CHECKED, "libdispatch_gpu_checked.so")
ROOT = os.path.dirname(PKG)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
SOURCES = [
    ("dsp_host.cu", ["-fmad=false"]),
    ("dsp_noalloc.cu", ["-fmad=false"]),
]
# floating-point flags of each precision code: FP64 without contraction
# (parity with the oracle), FP32 with fast division and square root, FP64
# with fused multiply-adds
PREC_FLAGS = {0: ["-fmad=false"], 1: ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"], 2: []}


def variants(checked=False):
    """Rows of csrc/dsp_variants.h: (id, type, tx, ty, nt, mb, precision,
    riemann, nonideal) of the full list, or of the bounds-checked build's."""
    txt = open(os.path.join(CSRC, "dsp_variants.h")).read()
    a = txt.index("#define DSP_VARIANT_LIST_ALL(X)")
    b = txt.index("#define DSP_VARIANT_LIST_CHECKED(X)")
    c = txt.index("#ifdef DSP_BOUNDS_CHECK")
    txt = txt[b:c] if checked else txt[a:b]
    rows = re.findall(r"X\((\d+),\s*(\w+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", txt)
    return [(int(a), b, int(c), int(d), int(e), int(f), int(g), int(r), int(n)) for a, b, c, d, e, f, g, r, n in rows]


def units(checked=False):
    out = [(src, src.replace(".cu", ".o"), flags) for src, flags in SOURCES]
    for vid, t, tx, ty, nt, mb, prec, rs, ni in variants(checked):
        defs = ["-DV_ID=%d" % vid, "-DV_T=%s" % t, "-DV_TX=%d" % tx, "-DV_TY=%d" % ty, "-DV_NT=%d" % nt,
                "-DV_MB=%d" % mb, "-DV_PREC=%d" % prec, "-DV_RS=%d" % rs, "-DV_NI=%d" % ni]
        out.append(("dsp_variant.cu", "dsp_variant_%d.o" % vid, defs + PREC_FLAGS[prec]))
    return out


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "dispatch.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(checked=False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra=(), checked=False) -> str:
    lib = LIB_CHECKED if checked else LIB
    out_dir = OUT_DIR_CHECKED if checked else OUT_DIR
    if checked:
        extra = tuple(extra) + ("-DDSP_BOUNDS_CHECK",)
    if not force and up_to_date(checked):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src, oname, flags in units(checked):
        obj = os.path.join(out_dir, oname)
        objs.append(obj)
        cmd = [nvcc, *COMMON, *ARCH, *flags, *extra, "-I", os.path.join(ROOT, "include"), "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
