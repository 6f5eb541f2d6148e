"""GPU: the z-slab decomposition (``decomp.py``) driving the CUDA library.
One rank on a periodic box exchanges its ghost planes with itself through
fish_get_planes / fish_set_planes on device memory and must give the
single-box result: bitwise in FP64 (built without multiply-add contraction),
within 2e-6 of each field's largest magnitude in FP32, where a cell may sit
in the march prologue of one box and the steady loop of the other and the
compiler may contract the two instantiations differently.  Ranks on several GPUs are covered by the gloo tests on
CPU; on one GPU the multi-rank exchange is not run."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_rank_slab_equals_single_box(F, precision):
    import torch
    from paper_0910_2854_gb300 import decomp
    w = W.random_smooth(24, 20, 18, seed=91, h=(0.04, 0.05, 0.055))
    nx, ny, nz = w.dims
    k0, nk, lo, hi = decomp.slab_extent(nz, 0, 1, True)
    assert (k0, nk, lo, hi) == (0, nz, decomp.HALO, decomp.HALO)
    st = np.zeros((8, lo + nk + hi, ny, nx))
    st[:, lo:lo + nk] = w.state
    box = F.Box(nx, ny, lo + nk + hi, w.gamma, precision=precision, h=w.h)
    box.set_state(st)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    run = decomp.SlabRun(box, nx, ny, nz, 0, 1, periodic=True, dist=None, device="cuda", dtype=dtype)
    ref = F.Box(*w.dims, w.gamma, precision=precision, h=w.h)
    ref.set_state(w.state)
    for _ in range(3):
        dt = run.step_cfl(0.5, 1)
        want = ref.cfl_dt(0.5)
        assert dt == want if precision == "fp64" else abs(dt - want) <= 1e-6 * want
        ref.step(dt)
    got, exp = box.get_state()[:, lo:lo + nk], ref.get_state()
    if precision == "fp64":
        assert np.array_equal(got, exp)
    else:
        scale = np.max(np.abs(exp), axis=(1, 2, 3), keepdims=True)
        assert float(np.max(np.abs(got - exp) / scale)) <= 2e-6
    box.close()
    ref.close()
