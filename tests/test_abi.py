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
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", offsetof(dsp_params, base_cells),
         offsetof(dsp_params, sched_capacity), offsetof(dsp_stats, status), offsetof(dsp_params, wait_budget),
         offsetof(dsp_params, variant), offsetof(dsp_params, riemann), offsetof(dsp_params, eta),
         offsetof(dsp_params, time_order));
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
                    D.dsp_params.wait_budget.offset, D.dsp_params.variant.offset, D.dsp_params.riemann.offset,
                    D.dsp_params.eta.offset, D.dsp_params.time_order.offset]


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle; the binding raises if the
    library is missing instead of computing anything itself."""
    pkg = os.path.join(ROOT, "paper_1705_10774_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith(".py"):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), fn


def test_layout_rules_are_checked_on_the_host():
    """dsp_create rejects bad layouts before touching the device: a level-1
    patch with an odd origin or size, overlapping level-1 patches, a level-0
    set that does not tile the box, a level other than 0 and 1, and two
    levels with the ready-queue dispatcher."""
    import numpy as np
    from paper_1705_10774_gb300 import ics
    coarse = ics.cartesian(2, 8)
    kw = dict(gamma=5 / 3, cfl=0.4, base_cells=coarse.base_cells, box_len=coarse.box_len)

    def code(n, lo, level, **extra):
        with __import__("pytest").raises(D.DispatchError) as e:
            D.Dispatch(n, lo, level=level, **kw, **extra)
        return e.value.code

    two = ics.two_level(coarse, 4, 8, fine_patch=8)
    lo_odd = two.lo.copy()
    lo_odd[-1, 0] += 1
    assert code(two.n, lo_odd, two.levels) == D.DSP_ERR_INVALID_ARG
    lo_ovl = two.lo.copy()
    lo_ovl[-1] = lo_ovl[-2]
    assert code(two.n, lo_ovl, two.levels) == D.DSP_ERR_INVALID_ARG
    assert code(coarse.n[:-1], coarse.lo[:-1], None) == D.DSP_ERR_INVALID_ARG
    lev2 = two.levels.copy()
    lev2[-1] = 2
    assert code(two.n, two.lo, lev2) == D.DSP_ERR_UNSUPPORTED
    assert code(two.n, two.lo, two.levels, dispatcher=0, time_mode=1) == D.DSP_ERR_UNSUPPORTED
    assert code(np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int64), None) == D.DSP_ERR_INVALID_ARG  # empty
    n_odd = two.n.copy()
    n_odd[-1] = (7, 8, 8)
    assert code(n_odd, two.lo, two.levels) == D.DSP_ERR_INVALID_ARG


def test_parameters_are_checked_on_the_host():
    """dsp_create rejects bad physics and dispatcher parameters before
    touching the device: grace outside [0, 1) or with the ready queue, an
    unknown time order or Riemann solver, too many slices, quadratic
    extrapolation with three slices, negative non-ideal coefficients or
    factors, an ambipolar term without ion density, and a variant id of the
    wrong solver or physics."""
    from paper_1705_10774_gb300 import ics
    lay = ics.cartesian(2, 8)
    kw = dict(gamma=5 / 3, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len, time_mode=1)

    def code(**extra):
        with __import__("pytest").raises(D.DispatchError) as e:
            D.Dispatch(lay.n, lay.lo, **kw, **extra)
        return e.value.code

    INV, UNS = D.DSP_ERR_INVALID_ARG, D.DSP_ERR_UNSUPPORTED
    assert code(grace=1.0) == INV
    assert code(grace=-0.1) == INV
    assert code(grace=0.3, dispatcher=0) == UNS
    assert code(time_order=3) == INV
    assert code(nslices=17) == INV
    assert code(grace=0.3, time_order=2, nslices=3) == INV
    assert code(riemann=2) == INV
    assert code(eta=-1.0) == INV
    assert code(gamma_ad=-1.0) == INV
    assert code(gamma_ad=2.0, rho_i=0.0) == INV
    assert code(eta=0.1, c_ohm=-1.0) == INV
    assert code(riemann=1, variant=0) == INV        # an HLL variant
    assert code(eta=0.1, variant=2) == INV          # an ideal-MHD variant


def test_noalloc_binding_refuses_arrays_it_cannot_vouch_for():
    """diagnostics_noalloc hands raw pointers to the library, which cannot
    tell a host array, a short array or a mixed dtype from a valid one: the
    binding must refuse them before any call reaches the device."""
    import numpy as np
    torch = pytest.importorskip("torch")
    n, npatch = (2, 3, 4), 2
    sizes = [npatch * 5 * 24, npatch * 3 * 3 * 4, npatch * 2 * 4 * 4, npatch * 2 * 3 * 5]
    host = [np.zeros(s) for s in sizes]
    with pytest.raises(ValueError, match="torch CUDA tensor"):
        D.diagnostics_noalloc(*host, npatch=npatch, n=n, dx=0.1)
    cpu = [torch.zeros(s, dtype=torch.float64) for s in sizes]
    with pytest.raises(ValueError, match="CUDA device"):
        D.diagnostics_noalloc(*cpu, npatch=npatch, n=n, dx=0.1)
    with pytest.raises(ValueError, match="every n"):
        D.diagnostics_noalloc(*cpu, npatch=npatch, n=(0, 3, 4), dx=0.1)


def test_bounds_checked_library_exports_every_declared_symbol():
    """The bounds-checked build (-DDSP_BOUNDS_CHECK, three variants) links and
    exports the same calls."""
    path = B.build(checked=True)
    lib = ctypes.CDLL(path)
    for name in declared():
        assert hasattr(lib, name), name
    assert [v[0] for v in B.variants(checked=True)] == [0, 2, 5]
