"""The z-slab decomposition of one box over several ranks (paper Sec. 3,
cuboid decomposition reduced to slabs; ``paper_0910_2854_gb300/decomp.py``)
on CPU: two gloo ranks, each advancing its slab plus ghost planes, must give
bitwise the single-box result in FP64 -- states and CFL time steps -- for
periodic and outflow boundaries.  The per-rank arithmetic is the FP64 oracle
behind the same box interface the CUDA library offers (apply, get_planes,
set_planes, cfl_dt_planes): what is tested here is the host side of the
decomposition -- slab bounds, ghost exchange (direction pairing, the
periodic ring, no ghost planes at outflow edges), the operator sequence
and the all-reduced time step."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class OracleSlabBox:
    """The oracle with the box interface SlabRun drives (host arrays)."""

    def __init__(self, oracle, nx, ny, nzl, gamma, bc, h):
        self.ob = oracle.OracleBox(nx, ny, nzl, gamma, bc=bc, h=h)
        self.n = (nx, ny, nzl)

    def apply(self, op, d, dt):
        (self.ob.fluid if op == 0 else self.ob.ct)(d, dt)

    def get_planes(self, k0, nk, out):
        out.view(-1).numpy()[:] = self.ob.state[:, k0:k0 + nk].reshape(-1)
        return out

    def set_planes(self, k0, nk, src):
        nx, ny, _ = self.n
        self.ob.state[:, k0:k0 + nk] = src.view(-1).numpy().reshape(8, nk, ny, nx)

    def cfl_dt_planes(self, k, k0, nk):
        return self.ob.cfl_planes(k, k0, nk)

    def sync(self):
        pass


def _case(bc):
    from paper_0910_2854_gb300 import workloads as W
    return W.random_smooth(12, 10, 19, seed=81, bc=bc, h=(0.08, 0.09, 0.05))


def _rank(rank, world, port, bc, steps, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_0910_2854_gb300 import decomp
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _case(bc)
        nx, ny, nz = w.dims
        k0, nk, lo, hi = decomp.slab_extent(nz, rank, world, bc == 0)
        box = OracleSlabBox(oracle, nx, ny, lo + nk + hi, w.gamma, w.bc, w.h)
        box.ob.state[:, lo:lo + nk] = w.state[:, k0:k0 + nk]
        run = decomp.SlabRun(box, nx, ny, nz, rank, world, periodic=(bc == 0), dist=dist, device="cpu",
                             dtype=torch.float64)
        dts = [run.step_cfl(0.5, 1) for _ in range(steps)]
        q.put((rank, k0, nk, box.ob.state[:, lo:lo + nk].copy(), dts, run.exchanges))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("bc", [0, 1])
def test_two_slabs_equal_the_single_box(bc):
    _run_and_compare(bc, 2, 2)


def _run_and_compare(bc, world, steps):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, bc, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    w = _case(bc)
    ob = oracle.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h)
    ob.set_state(w.state)
    want_dts = []
    for _ in range(steps):
        want_dts.append(ob.cfl(0.5))
        ob.step(want_dts[-1])
    got = np.empty_like(ob.state)
    for rank, k0, nk, st, dts, nex in res:
        assert dts == want_dts, (rank, dts, want_dts)
        assert nex == steps * 13  # one exchange per operator and one per CFL
        got[:, k0:k0 + nk] = st
    assert np.array_equal(got, ob.state), float(np.max(np.abs(got - ob.state)))


@pytest.mark.parametrize("bc", [0, 1])
def test_three_slabs_equal_the_single_box(bc):
    """Three ranks: a middle slab with neighbours on both sides."""
    _run_and_compare(bc, 3, 1)


def test_slab_bounds_cover_the_box():
    from paper_0910_2854_gb300.decomp import slab_bounds
    for nz, world in ((19, 2), (1024, 8), (10, 3), (7, 7)):
        spans = [slab_bounds(nz, r, world) for r in range(world)]
        assert spans[0][0] == 0 and sum(nk for _, nk in spans) == nz
        assert all(a[0] + a[1] == b[0] for a, b in zip(spans, spans[1:]))
        assert max(nk for _, nk in spans) - min(nk for _, nk in spans) <= 1
