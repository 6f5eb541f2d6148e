"""GPU test of fish_diagnostics_noalloc, the entry point for callers that
cannot let the library allocate device memory (host codes that manage all
device memory themselves, or loops where a cudaMalloc is not allowed).

It is called through the C ABI on device-resident states and must give what
fish_diagnostics gives for the same state, on consecutive calls that share
its fixed scratch array -- a box with as many z-planes as the array has
rows, then boxes with fewer z-planes than the one before, so that stale
rows would show.  Tolerances: each total
to 1e-12 of the sum of |values| times the cell volume (the two entry points
add in different orders), max |div b| to 1e-12 of max|b| / min(h).  Kept in
a file of its own that runs last."""
import ctypes

import numpy as np
import pytest

from paper_0910_2854_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available()
    from paper_0910_2854_gb300 import build
    build.build()
    import paper_0910_2854_gb300 as mod
    mod.load()
    return mod


def _reference_and_state(F, w, precision, steps):
    import torch
    box = F.Box(*w.dims, w.gamma, bc=w.bc, precision=precision, h=w.h)
    box.set_state(w.state)
    if steps:
        box.step_cfl(0.5, steps)
    ref = box.diagnostics()
    dt = torch.float64 if precision == "fp64" else torch.float32
    st = torch.empty(8 * w.ncells, dtype=dt, device="cuda")
    box.get_state_device(st)
    box.close()
    return ref, st


def _check(ref, got, st, h):
    # totals: 1e-12 of the sum of |values| times the cell volume (the sums
    # run in a different order); max |div b|: 1e-12 of max|b| / min(h)
    mag = st.view(8, -1).double().abs().sum(dim=1).cpu().numpy() * float(np.prod(h))
    assert np.all(np.abs(got[:8] - ref[:8]) <= 1e-12 * mag), (got, ref)
    bscale = float(st.view(8, -1)[5:].abs().max()) / min(h)
    assert abs(got[8] - ref[8]) <= 1e-12 * bscale, (got[8], ref[8])


def test_noalloc_diagnostics_match_existing_entry_point(F):
    import torch
    cases = [
        (W.random_smooth(24, 20, 18, seed=21, h=(0.04, 0.05, 0.055)), "fp64", 2),
        # as many z-planes as the scratch array has rows
        (W.random_smooth(4, 4, 4096, seed=24), "fp32", 1),
        (W.random_smooth(16, 12, 10, seed=22, bc=W.BC_OUTFLOW), "fp32", 3),
        (W.random_smooth(20, 16, 12, seed=23), "fp32", 2),
    ]
    stream = torch.cuda.current_stream()
    for w, prec, steps in cases:
        ref, st = _reference_and_state(F, w, prec, steps)
        out = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
        F.diagnostics_noalloc(st, w.dims, w.bc, w.h, out, stream)
        stream.synchronize()
        _check(ref, out.cpu().numpy(), st, w.h)


def test_noalloc_rejects_more_planes_than_its_scratch(F):
    import torch
    lib = F.load()
    st = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(9, dtype=torch.float64, device="cuda")
    code = lib.fish_diagnostics_noalloc(ctypes.c_void_p(st.data_ptr()), F.FISH_F64, 1, 1, 4097, 0, 1.0, 1.0,
                                        1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert code == F.FISH_ERR_ARG
    code = lib.fish_diagnostics_noalloc(None, F.FISH_F64, 1, 1, 1, 0, 1.0, 1.0, 1.0,
                                        ctypes.c_void_p(out.data_ptr()), None)
    assert code == F.FISH_ERR_ARG
