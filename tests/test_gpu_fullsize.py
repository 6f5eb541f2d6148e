"""Parity at the full size of the throughput workload: the 1024^3 FP32
turbulence box in the launch configuration bench.py times.  The oracle
cannot advance the whole box, but one directional operator changes a
pencil using only the pencils next to it, so for sampled pencils the oracle
advances the 3 x 3 bundle of pencils around each (periodic in the two
transverse directions, which leaves the central pencil exact) and the
central pencil is compared with the GPU result, 1e-5 relative per field."""
import numpy as np
import pytest

import oracle
from paper_0910_2854_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 1024
SAMPLES = [(0, 0), (511, 700), (1023, 1023), (37, 998)]


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    from paper_0910_2854_gb300 import build
    build.build()
    import paper_0910_2854_gb300 as F
    F.load()
    w = W.turbulence(N, device="cuda", dtype=torch.float32)
    box = F.Box(N, N, N, w.gamma, precision="fp32", h=w.h)
    box.set_state(w.state)
    dt = box.cfl_dt(0.5)
    st0 = w.state.reshape(8, N, N, N)
    out = torch.empty_like(w.state)
    yield F, torch, box, st0, out, w, dt
    box.close()


def bundle(torch, st, d, a, b):
    """The 3 x 3 bundle of pencils along axis d centred on transverse
    coordinates (a, b) of (d+1, d+2), as float64 numpy (8, nz, ny, nx)."""
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    idx = [None, None, None]
    idx[d] = torch.arange(N, device=st.device)
    idx[t1] = torch.tensor([(a - 1) % N, a, (a + 1) % N], device=st.device)
    idx[t2] = torch.tensor([(b - 1) % N, b, (b + 1) % N], device=st.device)
    # numpy order (z, y, x): tensor axis 3 - k for coordinate k; the two
    # transverse selections first, so no full-size copy is made
    sub = st
    for k in (t1, t2, d):
        sub = sub.index_select(3 - k, idx[k])
    return sub.double().cpu().numpy()


def centre(a, d):
    """The central pencil of a bundle array (8, nz, ny, nx)."""
    sl = [slice(None)] * 4
    for k in range(3):
        if k != d:
            sl[3 - k] = 1
    return a[tuple(sl)]


@pytest.mark.parametrize("op", ["fluid", "ct"])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_full_size_operator_on_sampled_pencils(setup, op, d):
    F, torch, box, st0, out, w, dt = setup
    box.set_state(st0.reshape(-1))
    box.apply(F.FISH_OP_FLUID if op == "fluid" else F.FISH_OP_CT, d, dt)
    box.get_state_device(out)
    got_all = out.reshape(8, N, N, N)
    for a, b in SAMPLES:
        sub = bundle(torch, st0, d, a, b)
        dims = (sub.shape[3], sub.shape[2], sub.shape[1])
        ob = oracle.OracleBox(*dims, w.gamma, bc=w.bc, h=w.h)
        ob.set_state(sub)
        getattr(ob, op)(d, dt)
        ref = centre(ob.state, d)
        got = centre(bundle(torch, got_all, d, a, b), d)
        scale = np.maximum(np.max(np.abs(ref), axis=1, keepdims=True), 1e-30)
        err = float(np.max(np.abs(got - ref) / scale))
        assert err <= 1e-5, (op, d, a, b, err)
