"""The C-ABI library builds, loads and exports every entry point the public
header declares, and the Python binding's structures match the C layout.
No GPU is touched."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1705_10774_gb300 import build as B
from paper_1705_10774_gb300 import dispatch as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR_DIR = os.path.join(ROOT, "include")


def declared():
    names = []
    for fn in sorted(os.listdir(HDR_DIR)):
        if fn.endswith(".h"):
            txt = open(os.path.join(HDR_DIR, fn)).read()
            names += re.findall(r"DSP_API\s+[\w\s\*]*?\b(dsp_\w+)\s*\(", txt)
    return names


def test_header_declares_the_documented_calls():
    names = declared()
    for must in ("dsp_create", "dsp_set_state", "dsp_advance", "dsp_get_state"):
        assert must in names
    assert sorted(names) == sorted(D.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)", out))
    assert set(declared()) <= exported


def test_binding_struct_layout_matches_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "dispatch.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(dsp_patch_desc), sizeof(dsp_params), sizeof(dsp_stats),
         sizeof(dsp_sched_entry), sizeof(dsp_diag));
  printf("%zu %zu %zu %zu %zu\n", offsetof(dsp_params, base_cells), offsetof(dsp_params, sched_capacity),
         offsetof(dsp_stats, status), offsetof(dsp_params, wait_budget), offsetof(dsp_params, variant));
  return 0;
}
''')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", HDR_DIR, str(src), "-o", str(exe)])
    a, b = subprocess.check_output([str(exe)]).decode().split("\n")[:2]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(s) for s in (D.dsp_patch_desc, D.dsp_params, D.dsp_stats,
                                               D.dsp_sched_entry, D.dsp_diag)]
    assert offs == [D.dsp_params.base_cells.offset, D.dsp_params.sched_capacity.offset, D.dsp_stats.status.offset,
                    D.dsp_params.wait_budget.offset, D.dsp_params.variant.offset]


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle; the binding raises if the
    library is missing instead of computing anything itself."""
    pkg = os.path.join(ROOT, "paper_1705_10774_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith(".py"):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), fn
