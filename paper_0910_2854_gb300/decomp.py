"""One box split over several GPUs along z: the paper's cuboid decomposition
(Sec. 3) reduced to slabs, one per rank, with ghost slabs exchanged before
every directional operator.

Rank r owns the z-planes [k0_r, k0_r + nk_r) of the global box (balanced
split, every slab at least HALO planes) and advances a local box of
lo + nk_r + hi planes: lo ghost planes below its own and hi above.  Before
each operator of the double step (the Strang-symmetric x-y-z-z-y-x sequence
of L_d and B_d, eq0081-eq0082 with reading C-4) the ghost planes are
refilled from the neighbouring ranks' boundary planes (periodic: the ring
closes, rank 0 takes the last rank's top planes from below).  At an outflow
edge of the global box the slab has no ghost planes on that side (lo or hi
is 0) and the local box applies the zeroth-order extrapolation there itself,
exactly as the single box does (reading C-14: a ghost copies the boundary
cell whole, its lower face included, which ghost planes could not express).
HALO = 4 covers the reach of every operator along z (the fluid sweep reads
three cells and the lower face of the fourth, the constrained transport four
cells); the x and y sweeps reach one plane.  Ghost planes are overwritten
before every operator, so what an operator leaves in them is never read.
The CFL time step is the minimum over the ranks' own planes (an all-reduce).

The host side here only moves planes and drives the box's operators; the
arithmetic runs in the box (the CUDA library on a GPU).  The box needs:
apply(op, d, dt), get_planes(k0, nk, out), set_planes(k0, nk, src),
cfl_dt_planes(k, k0, nk) and sync(); the exchange uses torch.distributed
(NCCL on GPUs, gloo on CPU) point-to-point messages.
"""
from __future__ import annotations

HALO = 4
FLUID, CT = 0, 1
# time order of one double step (reading C-4)
DOUBLE_STEP = ((FLUID, 0), (CT, 0), (FLUID, 1), (CT, 1), (FLUID, 2), (CT, 2),
               (CT, 2), (FLUID, 2), (CT, 1), (FLUID, 1), (CT, 0), (FLUID, 0))


def slab_bounds(nz, rank, world):
    """(k0, nk) of rank's slab: nz planes split as evenly as possible."""
    base, extra = divmod(nz, world)
    k0 = rank * base + min(rank, extra)
    return k0, base + (1 if rank < extra else 0)


def slab_extent(nz, rank, world, periodic):
    """(k0, nk, lo, hi): the rank's slab and its ghost planes below / above
    (none at an outflow edge of the global box; a single periodic rank keeps
    both and exchanges with itself)."""
    k0, nk = slab_bounds(nz, rank, world)
    lo = HALO if periodic or rank > 0 else 0
    hi = HALO if periodic or rank < world - 1 else 0
    return k0, nk, lo, hi


class SlabRun:
    """The rank's part of a box of global extent nz along z.

    ``box``: the local box (nx, ny, lo + nk + hi) of slab_extent, already
    holding the rank's planes at [lo, lo + nk); ``periodic``: the global boundary condition
    along z; ``dist``: torch.distributed (initialised) or None for a single
    rank; ``device``: where the exchange buffers live ("cuda" or "cpu");
    ``dtype``: torch dtype of the box's precision."""

    def __init__(self, box, nx, ny, nz, rank, world, periodic, dist=None, device="cuda", dtype=None):
        import torch
        self.box, self.rank, self.world, self.periodic, self.dist = box, rank, world, periodic, dist
        self.k0, self.nk, self.lo, self.hi = slab_extent(nz, rank, world, periodic)
        if self.nk < HALO and (self.lo or self.hi):
            raise ValueError("slab of %d planes is thinner than the halo (%d)" % (self.nk, HALO))
        self.plane = nx * ny
        n = 8 * HALO * self.plane
        self._send_lo = torch.empty(n, dtype=dtype, device=device)
        self._send_hi = torch.empty(n, dtype=dtype, device=device)
        self._recv_lo = torch.empty(n, dtype=dtype, device=device)
        self._recv_hi = torch.empty(n, dtype=dtype, device=device)
        self.device = device
        self.exchanges = 0

    # -- ghost planes ---------------------------------------------------------
    def exchange(self):
        """Refill the ghost planes from the neighbours."""
        b, H, nk, lo, hi = self.box, HALO, self.nk, self.lo, self.hi
        if not lo and not hi:
            self.exchanges += 1
            return
        lo_edge, hi_edge = lo == 0, hi == 0
        # own boundary planes: the lowest HALO go down, the highest HALO go up
        if not lo_edge:
            b.get_planes(lo, H, self._send_lo)
        if not hi_edge:
            b.get_planes(lo + nk - H, H, self._send_hi)
        b.sync()
        if self.world == 1:
            if self.periodic:
                self._recv_lo.copy_(self._send_hi)
                self._recv_hi.copy_(self._send_lo)
        else:
            # every rank posts: send up, receive from below, send down,
            # receive from above.  Tags keep the two directions apart where a
            # library matches by tag (gloo); where it matches in order (NCCL),
            # the common posting order pairs them (with two ranks on a
            # periodic ring both neighbours are the same rank).
            d = self.dist
            up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
            ops = []
            if not hi_edge:
                ops.append(d.P2POp(d.isend, self._send_hi, up, tag=1))
            if not lo_edge:
                ops.append(d.P2POp(d.irecv, self._recv_lo, down, tag=1))
                ops.append(d.P2POp(d.isend, self._send_lo, down, tag=2))
            if not hi_edge:
                ops.append(d.P2POp(d.irecv, self._recv_hi, up, tag=2))
            if ops:
                for r in d.batch_isend_irecv(ops):
                    r.wait()
        if not lo_edge:
            b.set_planes(0, H, self._recv_lo)
        if not hi_edge:
            b.set_planes(lo + nk, H, self._recv_hi)
        self.exchanges += 1

    # -- the method --------------------------------------------------------------
    def cfl_dt(self, k):
        """eq0083-eq0084 over the whole box: the minimum over the ranks' own
        planes."""
        self.exchange()
        dt = self.box.cfl_dt_planes(k, self.lo, self.nk)
        if self.world > 1:
            import torch
            t = torch.tensor([dt], dtype=torch.float64, device=self.device)
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
            dt = float(t.item())
        return dt

    def step(self, dt, nsteps=1):
        """nsteps double steps with the time step dt (time advances 2 dt each)."""
        for _ in range(nsteps):
            for op, d in DOUBLE_STEP:
                self.exchange()
                self.box.apply(op, d, dt)

    def step_cfl(self, k, nsteps=1):
        """nsteps double steps, each with dt = k * CFL of the state at its
        start; returns the last dt."""
        dt = None
        for _ in range(nsteps):
            dt = self.cfl_dt(k)
            self.step(dt)
        return dt
