"""The allocation-free diagnostics entry point, through the C ABI.

dsp_diagnostics_noalloc serves callers that cannot call cudaMalloc (an
application whose device memory all belongs to its own pool allocator, or a
latency-sensitive loop that must not trigger cudaMalloc's device-wide
synchronisation).  It reads a state from the caller's device arrays (all
patches of one size and one cell size) and keeps its scratch in a fixed
device array inside the library.  It must agree with dsp_diagnostics of a
context holding the same state, and with exact numpy sums of the same values,
on two calls in a row (the second on a different state, so stale scratch
contents would show), and reject more patches than its scratch holds, no
patches, an empty axis and a non-positive cell size.  This file is collected
last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import (DSP_ERR_INVALID_ARG, DSP_NOALLOC_MAX_PATCHES, VP, Dispatch, DispatchError,
                                             diagnostics_noalloc, dsp_diag, load)

from test_oracle_diagnostics import expected


def close(a, b, scale):
    return abs(a - b) <= 1e-12 * scale


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("cells", [(16, 16, 16), (12, 10, 6)])
def test_noalloc_diagnostics_match_context_diagnostics_on_two_calls(precision, cells):
    lay = ics.cartesian(2, cells, dx=1.0 / (2 * cells[0]))
    rng = np.random.default_rng(5)
    X, Y, Z = lay.base_cells
    shape = (Z, Y, X)
    v = ics.solenoidal_velocity(shape, lay.box_len, 1.0, 3.0, 1.0, rng)
    f = ics.Fields(rho=np.ones(shape), v=v, p=np.full(shape, 0.6), bx=np.full(shape, 0.8), by=np.zeros(shape),
                   bz=np.zeros(shape), gamma=5.0 / 3.0)
    g = Dispatch(lay.n, lay.lo, gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                 precision=precision, time_mode=0)
    g.set_state(*ics.to_patches(lay, f))
    dtype = torch.float64 if precision == 0 else torch.float32
    for call in range(2):
        ref = g.diagnostics()
        dev = [torch.empty(s, dtype=dtype, device="cuda") for s in g.sizes]
        g.get_state(out=dev)
        torch.cuda.synchronize()
        got = diagnostics_noalloc(*dev, npatch=lay.npatch, n=cells, dx=lay.dx)
        scale = max(abs(ref["mass"]), abs(ref["energy"]), 1.0)
        assert close(got["mass"], ref["mass"], scale) and close(got["energy"], ref["energy"], scale)
        for d in range(3):
            assert close(got["mom"][d], ref["mom"][d], scale)
            assert close(got["bmean"][d], ref["bmean"][d], scale)
        assert got["max_divb"] == ref["max_divb"] and got["max_b"] == ref["max_b"]
        # against exact sums of the same values, independently of either kernel
        tot, sc, mdiv, mb = expected(lay, [a.double().cpu().numpy() for a in dev])
        flat = [got["mass"], *got["mom"], got["energy"], *got["bmean"]]
        for q in range(8):
            assert abs(flat[q] - tot[q]) <= 1e-13 * sc[q], q
        assert got["max_divb"] == mdiv and got["max_b"] == mb
        g.advance(max_sweeps=3)        # the second call sees a different state
    g.close()


def _raw(dev, npatch, n, dx):
    """The C entry point itself, past the binding's own checks."""
    nn = (ctypes.c_int32 * 3)(*n)
    d = dsp_diag()
    return load().dsp_diagnostics_noalloc(*[VP(a.data_ptr()) for a in dev], 0, npatch, nn, dx, VP(0),
                                          ctypes.byref(d))


def test_noalloc_rejects_more_patches_than_its_scratch_holds():
    npatch = DSP_NOALLOC_MAX_PATCHES + 1
    dev = [torch.zeros(npatch * k, dtype=torch.float64, device="cuda") for k in (5, 2, 2, 2)]
    with pytest.raises(DispatchError) as e:
        diagnostics_noalloc(*dev, npatch=npatch, n=(1, 1, 1), dx=0.1)
    assert e.value.code == DSP_ERR_INVALID_ARG


def test_noalloc_rejects_empty_and_degenerate_requests():
    dev = [torch.ones(8 * k, dtype=torch.float64, device="cuda") for k in (5, 2, 2, 2)]
    assert _raw(dev, 8, (1, 1, 1), 0.1) == 0
    assert _raw(dev, 0, (1, 1, 1), 0.1) == DSP_ERR_INVALID_ARG
    assert _raw(dev, 8, (0, 1, 1), 0.1) == DSP_ERR_INVALID_ARG
    assert _raw(dev, 8, (1, 1, -2), 0.1) == DSP_ERR_INVALID_ARG
    assert _raw(dev, 8, (1, 1, 1), 0.0) == DSP_ERR_INVALID_ARG
    assert _raw(dev, 8, (1, 1, 1), -0.1) == DSP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        diagnostics_noalloc(*dev, npatch=8, n=(2, 1, 1), dx=0.1)       # arrays too short for n
    with pytest.raises(ValueError):
        diagnostics_noalloc(dev[0], dev[1], dev[2], dev[3].float(), npatch=8, n=(1, 1, 1), dx=0.1)
