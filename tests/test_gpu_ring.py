"""GPU: the fluid sweep fed through the shared-memory ring of bulk copies
gives bitwise the result of the register-prefetch column march (same
arithmetic in the same order), for every direction, limiter and boundary,
for boxes whose fast extent is a multiple of four, including blocks that
cover only part of a row (fast extent not a multiple of 256) and pencils
shorter than the ring, and against the oracle on its own."""
import numpy as np
import pytest

import oracle
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


RING_BOXES = {
    "periodic": lambda: W.random_smooth(32, 24, 20, seed=71, h=(0.03, 0.04, 0.05)),
    # fast extent 260: one full block of 256 columns and one of 4 per row
    "partial_block": lambda: W.random_smooth(260, 8, 12, seed=72),
    "outflow": lambda: W.random_smooth(24, 20, 9, seed=73, bc=W.BC_OUTFLOW),
    # pencils of 1, 5 and 3 cells: fewer stages than the ring holds
    "short": lambda: W.random_smooth(8, 4, 5, seed=74),
    "single_layer": lambda: W.random_smooth(12, 8, 1, seed=75, bc=W.BC_OUTFLOW),
}


def boxes(F, w, **kw):
    out = []
    for k in ("ring", "column"):
        b = F.Box(*w.dims, w.gamma, bc=w.bc, precision="fp32", h=w.h, kernels=k, **kw)
        b.set_state(w.state)
        out.append(b)
    return out


@pytest.mark.parametrize("box", sorted(RING_BOXES))
@pytest.mark.parametrize("lim", [0, 1, 3])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_ring_fluid_bitwise(F, box, lim, d):
    w = RING_BOXES[box]()
    ring, col = boxes(F, w, limiter=lim)
    dt = 0.4 * col.cfl_dt(1.0)
    ring.fluid(d, dt)
    col.fluid(d, dt)
    a, b = ring.get_state(), col.get_state()
    assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
    ring.close()
    col.close()


@pytest.mark.parametrize("box", ["periodic", "outflow", "partial_block"])
def test_ring_graph_steps_bitwise(F, box):
    """Five graph-replayed double steps with the CFL reduced in the last x
    sweep: state and time step equal the column kernels' bitwise."""
    w = RING_BOXES[box]()
    ring, col = boxes(F, w)
    ring.step_cfl(0.5, 5)
    col.step_cfl(0.5, 5)
    assert ring.last_dt() == col.last_dt()
    assert np.array_equal(ring.get_state(), col.get_state())
    ring.close()
    col.close()


def test_ring_step_against_oracle(F):
    """The ring path on its own against the FP64 oracle after one double
    step (1e-5 relative to each field's largest magnitude, per cell)."""
    w = RING_BOXES["partial_block"]()
    ob = oracle.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h)
    ob.set_state(w.state)
    gb = F.Box(*w.dims, w.gamma, bc=w.bc, precision="fp32", h=w.h, kernels="ring")
    gb.set_state(w.state)
    dt = ob.cfl(0.5)
    ob.step(dt)
    gb.step(dt)
    got = gb.get_state()
    scale = np.maximum(np.max(np.abs(ob.state), axis=(1, 2, 3), keepdims=True), 1e-300)
    assert float(np.max(np.abs(got - ob.state) / scale)) <= 1e-5
    gb.close()
