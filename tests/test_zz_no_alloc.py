"""The allocation-free diagnostics entry point, through the C ABI.

dsp_diagnostics_noalloc serves callers that cannot call cudaMalloc (an
application whose device memory all belongs to its own pool allocator, or a
latency-sensitive loop that must not trigger cudaMalloc's device-wide
synchronisation).  It reads a state from the caller's device arrays and keeps
its scratch in a fixed device array inside the library.  It must agree with
dsp_diagnostics of a context holding the same state, on two calls in a row
(the second on a different state, so stale scratch contents would show), and
reject more patches than its scratch holds.  This file is collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_10774_gb300 import ics
from paper_1705_10774_gb300.dispatch import (DSP_ERR_INVALID_ARG, DSP_NOALLOC_MAX_PATCHES, Dispatch, DispatchError,
                                             diagnostics_noalloc)


def close(a, b, scale):
    return abs(a - b) <= 1e-12 * scale


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_diagnostics_match_context_diagnostics_on_two_calls(precision):
    lay, f = ics.config_turbulence(seed=5, patches=2, n=16, mach=1.0)
    g = Dispatch(lay.n, lay.lo, gamma=f.gamma, cfl=0.4, base_cells=lay.base_cells, box_len=lay.box_len,
                 precision=precision, time_mode=0)
    g.set_state(*ics.to_patches(lay, f))
    dtype = torch.float64 if precision == 0 else torch.float32
    for call in range(2):
        ref = g.diagnostics()
        dev = [torch.empty(s, dtype=dtype, device="cuda") for s in g.sizes]
        g.get_state(out=dev)
        torch.cuda.synchronize()
        got = diagnostics_noalloc(*dev, npatch=lay.npatch, n=lay.n[0], dx=lay.dx)
        scale = max(abs(ref["mass"]), abs(ref["energy"]), 1.0)
        assert close(got["mass"], ref["mass"], scale) and close(got["energy"], ref["energy"], scale)
        for d in range(3):
            assert close(got["mom"][d], ref["mom"][d], scale)
            assert close(got["bmean"][d], ref["bmean"][d], scale)
        assert got["max_divb"] == ref["max_divb"] and got["max_b"] == ref["max_b"]
        g.advance(max_sweeps=3)        # the second call sees a different state
    g.close()


def test_noalloc_rejects_more_patches_than_its_scratch_holds():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(DispatchError) as e:
        diagnostics_noalloc(x, x, x, x, npatch=DSP_NOALLOC_MAX_PATCHES + 1, n=(4, 4, 4), dx=0.1)
    assert e.value.code == DSP_ERR_INVALID_ARG
