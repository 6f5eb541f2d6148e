"""Seeded synthetic initial conditions for the FISH sweep (inputs only).

This module holds no arithmetic of the method: it only builds initial states
(cell-averaged rho, m, E and face-averaged b in the layout of the C ABI) for
the test problems of the paper (Sec. 4) and the throughput workloads.  Both
the CUDA path and the CPU oracle consume what it returns, so it imports
neither.

Layout of a state: float64 array (8, nz, ny, nx), x fastest; fields rho,
m_x, m_y, m_z, E, b_x (face i+1/2), b_y (face j+1/2), b_z (face k+1/2).
E = p/(gamma-1) + rho v^2/2 + b_c^2/2 with b_c the arithmetic mean of the two
faces of each cell (periodic wrap or clamped at outflow boundaries), so that
the gas pressure recovered by the solver equals the prescribed one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_PERIODIC, BC_OUTFLOW = 0, 1


@dataclass
class Workload:
    """An initial state plus the parameters a box needs."""
    name: str
    state: np.ndarray            # (8, nz, ny, nx) float64
    gamma: float
    h: tuple                     # (dx, dy, dz)
    bc: int = BC_PERIODIC
    phi: np.ndarray | None = None  # cell-centred potential (nz, ny, nx) or None
    meta: dict = field(default_factory=dict)

    @property
    def dims(self):
        return (self.state.shape[3], self.state.shape[2], self.state.shape[1])

    @property
    def ncells(self):
        return int(self.state.shape[1] * self.state.shape[2] * self.state.shape[3])


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def cell_centred(b_faces, bc):
    """Mean of the two faces of each cell along each axis (x, y, z)."""
    out = []
    for ax in range(3):
        b = b_faces[ax]
        npax = 2 - ax
        if bc == BC_PERIODIC:
            lo = np.roll(b, 1, axis=npax)
        else:
            n = b.shape[npax]
            sel = np.concatenate([[0], np.arange(n - 1)]).astype(np.int64)
            lo = np.take(b, sel, axis=npax)
        out.append(0.5 * (lo + b))
    return out


def assemble(rho, v, p, b_faces, gamma, bc):
    """State array from primitive cell values and face fields."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    vx, vy, vz = (np.broadcast_to(np.asarray(c, dtype=np.float64), shape) for c in v)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), shape)
    bf = [np.broadcast_to(np.asarray(c, dtype=np.float64), shape).copy() for c in b_faces]
    bcc = cell_centred(bf, bc)
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) \
        + 0.5 * (bcc[0] ** 2 + bcc[1] ** 2 + bcc[2] ** 2)
    st = np.empty((8,) + shape, dtype=np.float64)
    st[0] = rho
    st[1] = rho * vx
    st[2] = rho * vy
    st[3] = rho * vz
    st[4] = E
    st[5], st[6], st[7] = bf
    return st


def _grid(n, L=1.0, x0=0.0):
    """Cell centres, left faces and right faces of n cells on [x0, x0+L]."""
    h = L / n
    xl = x0 + h * np.arange(n)
    return xl + 0.5 * h, xl, xl + h, h


def _sin_avg(k, xl, xr):
    """Exact average of sin(k x) over [xl, xr]."""
    return (np.cos(k * xl) - np.cos(k * xr)) / (k * (xr - xl))


def _cos_avg(k, xl, xr):
    return (np.sin(k * xr) - np.sin(k * xl)) / (k * (xr - xl))


def _mesh(nx, ny, nz):
    return (nz, ny, nx)


# --------------------------------------------------------------------------
# circularly polarised Alfven wave (Sec. 4 "Circularly polarised Alfven waves")
# --------------------------------------------------------------------------

def alfven_x(nx, ny=None, nz=None, amp=0.1, gamma=5.0 / 3.0, p0=0.1):
    """Wave vector along x on [0,1]^3: rho = 1, p = 0.1, b_x = 1, v_x = 0,
    v_y = b_y = A sin(2 pi x), v_z = b_z = A cos(2 pi x); cell and face values
    are exact averages of the sines.  The wave returns to its initial state
    after t = 1 (v_A = b_par / sqrt(rho) = 1)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    _, xl, xr, hx = _grid(nx)
    k = 2.0 * math.pi
    s = _sin_avg(k, xl, xr)[None, None, :]
    c = _cos_avg(k, xl, xr)[None, None, :]
    shp = _mesh(nx, ny, nz)
    one = np.ones(shp)
    st = assemble(one, (0.0 * one, amp * s * one, amp * c * one), p0,
                  (one, amp * s * one, amp * c * one), gamma, BC_PERIODIC)
    return Workload("alfven_x", st, gamma, (hx, 1.0 / ny, 1.0 / nz), BC_PERIODIC,
                    meta={"amp": amp, "period": 1.0})


def alfven_oblique(N, alpha_deg=30.0, amp=0.1, gamma=5.0 / 3.0, p0=0.1):
    """The paper's 2-D test: propagation at angle alpha to x on
    [0, 1/cos a] x [0, 1/sin a] with N x N x 1 cells.  b comes from the edge
    vector potential A_z = y cos a - x sin a + A cos(2 pi xi)/(2 pi),
    xi = x cos a + y sin a, so the discrete divergence vanishes; b_z and the
    velocities are exact cell averages."""
    a = math.radians(alpha_deg)
    ca, sa = math.cos(a), math.sin(a)
    Lx, Ly = 1.0 / ca, 1.0 / sa
    hx, hy = Lx / N, Ly / N
    k = 2.0 * math.pi
    xf = hx * np.arange(N + 1)          # faces x_{i-1/2}, i = 0..N
    yf = hy * np.arange(N + 1)
    xc = 0.5 * (xf[:-1] + xf[1:])
    yc = 0.5 * (yf[:-1] + yf[1:])

    def Az(x, y):
        return y * ca - x * sa + amp * np.cos(k * (x * ca + y * sa)) / k

    # b_x at (x_{i+1/2}, y_j): [A_z(x_{i+1/2}, y_{j+1/2}) - A_z(x_{i+1/2}, y_{j-1/2})]/hy
    X, Yt = np.meshgrid(xf[1:], yf[1:], indexing="xy")
    _, Yb = np.meshgrid(xf[1:], yf[:-1], indexing="xy")
    bx = (Az(X, Yt) - Az(X, Yb)) / hy
    # b_y at (x_i, y_{j+1/2}): -[A_z(x_{i+1/2}, y_{j+1/2}) - A_z(x_{i-1/2}, y_{j+1/2})]/hx
    Xr, Y = np.meshgrid(xf[1:], yf[1:], indexing="xy")
    Xl, _ = np.meshgrid(xf[:-1], yf[1:], indexing="xy")
    by = -(Az(Xr, Y) - Az(Xl, Y)) / hx
    # cell averages of sin/cos(2 pi xi): separable sinc factors
    fx = math.sin(k * ca * hx / 2) / (k * ca * hx / 2)
    fy = math.sin(k * sa * hy / 2) / (k * sa * hy / 2)
    XC, YC = np.meshgrid(xc, yc, indexing="xy")
    ph = k * (XC * ca + YC * sa)
    s = np.sin(ph) * fx * fy
    c = np.cos(ph) * fx * fy
    vperp, vz = amp * s, amp * c
    vx = -sa * vperp
    vy = ca * vperp
    bz = amp * c
    one = np.ones((1, N, N))
    st = assemble(one, (vx[None], vy[None], vz[None]), p0,
                  (bx[None], by[None], bz[None]), gamma, BC_PERIODIC)
    return Workload("alfven_oblique", st, gamma, (hx, hy, 1.0), BC_PERIODIC,
                    meta={"amp": amp, "period": 1.0, "alpha": alpha_deg})


def fast_wave(n, eps=1e-6, rho0=1.0, p0=0.6, bx=0.8, by=0.6, gamma=5.0 / 3.0):
    """Linear fast magnetosonic wave along x on [0,1] (n x 1 x 1 cells):
    background rho0, p0, b = (bx, by, 0) at rest; perturbation eps sin(2 pi x)
    along the textbook right eigenvector of 1-D ideal MHD for the fast speed
    c^2 = ((a^2 + B^2) + sqrt((a^2 + B^2)^2 - 4 a^2 bx^2)) / 2 (units with
    rho0 = 1 absorbed), a^2 = gamma p0 / rho0, B^2 = (bx^2 + by^2)/rho0:
      dvx = eps s, drho = rho0 dvx / c, dp = gamma p0 dvx / c,
      dby = by rho0 c dvx / (c^2 rho0 - bx^2), dvy = -bx dby / (c rho0).
    It travels at +c, so after t = 1/c it returns to the initial state up to
    O(eps^2)."""
    a2 = gamma * p0 / rho0
    B2 = (bx * bx + by * by) / rho0
    c = math.sqrt(0.5 * ((a2 + B2) + math.sqrt((a2 + B2) ** 2 - 4 * a2 * bx * bx / rho0)))
    _, xl, xr, h = _grid(n)
    s = _sin_avg(2 * math.pi, xl, xr)
    dvx = eps * s
    drho = rho0 * dvx / c
    dp = gamma * p0 * dvx / c
    dby = by * rho0 * c * dvx / (c * c * rho0 - bx * bx)
    dvy = -bx * dby / (c * rho0)
    one = np.ones((1, 1, n))
    st = assemble((rho0 + drho)[None, None] * one, (dvx[None, None] * one, dvy[None, None] * one, 0 * one),
                  (p0 + dp)[None, None] * one, (bx * one, (by + dby)[None, None] * one, 0 * one),
                  gamma, BC_PERIODIC)
    return Workload("fast_wave", st, gamma, (h, 1.0, 1.0), BC_PERIODIC,
                    meta={"c": c, "eps": eps, "period": 1.0 / c})


# --------------------------------------------------------------------------
# smooth advection, shock tubes
# --------------------------------------------------------------------------

def entropy_wave(n, axis=0, ntrans=4, amp=0.2, vel=1.0, gamma=5.0 / 3.0):
    """rho = 1 + A sin(2 pi s) (exact cell averages) advected at uniform
    velocity ``vel`` along ``axis`` with uniform pressure 1 and b = 0; the exact
    solution is the translated profile."""
    _, xl, xr, h = _grid(n)
    prof = 1.0 + amp * _sin_avg(2 * math.pi, xl, xr)
    dims = [ntrans, ntrans, ntrans]
    dims[axis] = n
    nx, ny, nz = dims
    shape = _mesh(nx, ny, nz)
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    rho = np.broadcast_to(prof[tuple(sl)], shape).copy()
    v = [0.0, 0.0, 0.0]
    v[axis] = vel
    zero = np.zeros(shape)
    st = assemble(rho, tuple(vv + zero for vv in v), 1.0, (zero, zero, zero), gamma, BC_PERIODIC)
    hh = [1.0 / nx, 1.0 / ny, 1.0 / nz]
    return Workload("entropy_wave", st, gamma, tuple(hh), BC_PERIODIC,
                    meta={"axis": axis, "amp": amp, "vel": vel})


def shock_tube(n, axis=0, ntrans=4, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1),
               gamma=1.4, b_n=0.0, b_t=(0.0, 0.0), name="sod", mirror=False):
    """1-D Riemann problem (rho, u, p) on [0,1] along ``axis`` with the jump at
    0.5, uniform across the transverse axes, outflow boundaries.  Magnetic
    field: normal component b_n everywhere, first transverse component
    +b_t[0] on the left and b_t[1] on the right (Brio-Wu style)."""
    dims = [ntrans, ntrans, ntrans]
    dims[axis] = n
    nx, ny, nz = dims
    shape = _mesh(nx, ny, nz)
    xc, _, _, h = _grid(n)
    L = xc < 0.5
    if mirror:
        L = xc > 0.5
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    Lm = np.broadcast_to(L[tuple(sl)], shape)
    rho = np.where(Lm, left[0], right[0])
    un = np.where(Lm, left[1], right[1])
    p = np.where(Lm, left[2], right[2])
    bt = np.where(Lm, b_t[0], b_t[1])
    if mirror:
        un = -un
    v = [np.zeros(shape)] * 3
    v = [np.zeros(shape), np.zeros(shape), np.zeros(shape)]
    v[axis] = un
    b = [np.zeros(shape), np.zeros(shape), np.zeros(shape)]
    b[axis] = b_n + np.zeros(shape)
    b[(axis + 1) % 3] = bt
    st = assemble(rho, tuple(v), p, tuple(b), gamma, BC_OUTFLOW)
    hh = [1.0 / nx, 1.0 / ny, 1.0 / nz]
    return Workload(name, st, gamma, tuple(hh), BC_OUTFLOW,
                    meta={"axis": axis, "left": left, "right": right})


def sod(n, axis=0, ntrans=4, mirror=False):
    return shock_tube(n, axis, ntrans, mirror=mirror)


def brio_wu(n, axis=0, ntrans=4):
    """Brio-Wu MHD tube: gamma = 2, rho 1/0.125, p 1/0.1, b_n = 0.75,
    b_t = +1 / -1."""
    return shock_tube(n, axis, ntrans, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1),
                      gamma=2.0, b_n=0.75, b_t=(1.0, -1.0), name="brio_wu")


# --------------------------------------------------------------------------
# 3-D workloads
# --------------------------------------------------------------------------

def orszag_tang(n, gamma=5.0 / 3.0):
    """3-D Orszag-Tang-type vortex on [0,1]^3: rho = 25/(36 pi), p = 5/(12 pi),
    v = (-sin 2pi y, sin 2pi x, 0.1 sin 2pi z) at cell centres,
    b = (-sin 2pi y, sin 4pi x, 0)/sqrt(4 pi) sampled at face centres (b_x
    depends on y only and b_y on x only, so the discrete divergence is 0)."""
    xc, _, _, h = _grid(n)
    k = 2 * math.pi
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    rho = np.full(X.shape, 25.0 / (36.0 * math.pi))
    p = 5.0 / (12.0 * math.pi)
    v = (-np.sin(k * Y), np.sin(k * X), 0.1 * np.sin(k * Z))
    s4 = 1.0 / math.sqrt(4 * math.pi)
    bx = -np.sin(k * Y) * s4
    by = np.sin(2 * k * X) * s4
    bz = np.zeros(X.shape)
    st = assemble(rho, v, p, (bx, by, bz), gamma, BC_PERIODIC)
    return Workload("orszag_tang", st, gamma, (h, h, h), BC_PERIODIC)


def random_smooth(nx, ny, nz, seed=0, gamma=5.0 / 3.0, vamp=0.3, bamp=0.1, bmean=(0.2, 0.1, 0.05),
                  h=None, bc=BC_PERIODIC):
    """Seeded smooth periodic state with a few random Fourier modes: positive
    rho and p, velocities ~ vamp, b = mean + curl of an edge vector potential
    (discretely divergence-free)."""
    rng = np.random.RandomState(seed)
    if h is None:
        h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    hx, hy, hz = h
    Lx, Ly, Lz = nx * hx, ny * hy, nz * hz
    ic = np.arange(nx) + 0.5
    jc = np.arange(ny) + 0.5
    kc = np.arange(nz) + 0.5

    def modes(xs, ys, zs, amp, nm=4):
        Z, Y, X = np.meshgrid(zs * hz / Lz, ys * hy / Ly, xs * hx / Lx, indexing="ij")
        f = np.zeros(X.shape)
        for _ in range(nm):
            kx, ky, kz = rng.randint(-2, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(0.3, 1.0) * amp
            f += a * np.sin(2 * math.pi * (kx * X + ky * Y + kz * Z) + ph)
        return f

    rho = 1.0 + modes(ic, jc, kc, 0.15)
    p = 1.0 + modes(ic, jc, kc, 0.15)
    v = tuple(modes(ic, jc, kc, vamp) for _ in range(3))
    # edge potentials: A_x at (i, j+1/2, k+1/2), A_y at (i+1/2, j, k+1/2), A_z at (i+1/2, j+1/2, k)
    Ax = modes(ic, jc + 0.5, kc + 0.5, bamp * hx * nx / (2 * math.pi))
    Ay = modes(ic + 0.5, jc, kc + 0.5, bamp * hy * ny / (2 * math.pi))
    Azp = modes(ic + 0.5, jc + 0.5, kc, bamp * hz * nz / (2 * math.pi))

    def dm(a, axis):  # a[c] - a[c-1] along numpy axis (periodic)
        return a - np.roll(a, 1, axis=axis)

    bx = bmean[0] + dm(Azp, 1) / hy - dm(Ay, 0) / hz
    by = bmean[1] + dm(Ax, 0) / hz - dm(Azp, 2) / hx
    bz = bmean[2] + dm(Ay, 2) / hx - dm(Ax, 1) / hy
    st = assemble(rho, v, p, (bx, by, bz), gamma, bc)
    return Workload("random_smooth", st, gamma, tuple(h), bc, meta={"seed": seed})


def blast(nx, ny, nz, gamma=5.0 / 3.0, p_in=100.0, p_out=1.0, b=(1.0, 0.0, 0.0), radius_frac=0.1,
          bc=BC_PERIODIC, centre=(0.5, 0.5, 0.5)):
    """Spherical blast: rho = 1, v = 0, p = p_in inside r < radius_frac times
    the shortest box side, p_out outside, uniform b, unit cells scaled so the
    longest side has length 1.  ``centre``: position of the centre as a
    fraction of each side (the default centres the blast, which makes the
    flow mirror-symmetric about the box's mid-planes)."""
    L = float(max(nx, ny, nz))
    h = 1.0 / L
    xs = (np.arange(nx) + 0.5) * h - centre[0] * nx * h
    ys = (np.arange(ny) + 0.5) * h - centre[1] * ny * h
    zs = (np.arange(nz) + 0.5) * h - centre[2] * nz * h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    R = radius_frac * min(nx, ny, nz) * h
    p = np.where(r < R, p_in, p_out)
    one = np.ones(X.shape)
    st = assemble(one, (0 * one, 0 * one, 0 * one), p, tuple(c * one for c in b), gamma, bc)
    return Workload("blast", st, gamma, (h, h, h), bc)


def polytrope(n, half_width=1.45, rho_c=1.0, R=1.0, atm=1e-3, gamma=2.0):
    """n = 1 polytrope in hydrostatic equilibrium (G = 1): rho = rho_c sin(x)/x,
    x = pi r/R, p = K rho^2 with K = 2 R^2 / pi (R = pi sqrt(K/(2 pi))), fixed
    analytic potential phi = -2 K rho(r) - M/R inside and -M/r outside,
    M = 4 R^3 rho_c / pi; atmosphere rho = atm rho_c with the sound speed of
    the centre, p = atm K rho_c^2; box [-w, w]^3, outflow.  With a thinner or
    colder atmosphere (1e-6 rho_c, p = K rho^2) the surface pressure of the
    analytic profile drives a shock into it at ~30 times the initial CFL
    speed within the first step."""
    K = 2.0 * R * R / math.pi
    M = 4.0 * R ** 3 * rho_c / math.pi
    h = 2.0 * half_width / n
    xs = -half_width + (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    x = math.pi * r / R
    with np.errstate(invalid="ignore", divide="ignore"):
        prof = np.where(x > 0, np.sin(x) / np.where(x > 0, x, 1.0), 1.0)
    inside = r < R
    rho_in = rho_c * prof
    rho = np.where(inside, np.maximum(rho_in, atm * rho_c), atm * rho_c)
    p = np.maximum(K * rho * rho, atm * K * rho_c * rho_c)
    phi = np.where(inside, -2.0 * K * rho_c * prof - M / R, -M / np.maximum(r, 1e-300))
    one = np.ones(X.shape)
    st = assemble(rho, (0 * one, 0 * one, 0 * one), p, (0 * one, 0 * one, 0 * one), gamma, BC_OUTFLOW)
    return Workload("polytrope", st, gamma, (h, h, h), BC_OUTFLOW, phi=phi,
                    meta={"K": K, "M": M, "rho_c": rho_c, "tau_hse": 0.5 / math.sqrt(3 * M / (4 * math.pi * R ** 3))})


# --------------------------------------------------------------------------
# random-phase MHD turbulence (k^-2 spectrum, |k| <= 8)
# --------------------------------------------------------------------------

def turbulence_coefficients(seed, kmax=8):
    """Complex Gaussian Fourier coefficients c_k, |c_k|^2 ~ k^-2 for
    1 <= |k| <= kmax (integer wave vectors), zero elsewhere.  Shape
    (3, 2kmax+1, 2kmax+1, 2kmax+1) indexed [comp, kz, ky, kx] + kmax."""
    rng = np.random.RandomState(seed)
    m = 2 * kmax + 1
    k1 = np.arange(m) - kmax
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    mask = (kk >= 1) & (kk <= kmax)
    amp = np.where(mask, 1.0 / np.where(kk > 0, kk, 1.0), 0.0)
    c = (rng.standard_normal((3, m, m, m)) + 1j * rng.standard_normal((3, m, m, m))) * amp[None]
    return c


def _synth(coef, pos_x, pos_y, pos_z, kmax, torch_device=None, chunk=64):
    """Real field sum_k Re(c_k exp(2 pi i k.x)) at the tensor-product points
    (pos in units of the box length).  Evaluated separably; with
    ``torch_device`` it runs on that device (chunked along z)."""
    k1 = np.arange(2 * kmax + 1) - kmax
    ex = np.exp(2j * math.pi * np.outer(pos_x, k1))   # (nx, m)
    ey = np.exp(2j * math.pi * np.outer(pos_y, k1))
    ez = np.exp(2j * math.pi * np.outer(pos_z, k1))
    if torch_device is None:
        t1 = np.einsum("abc,xc->abx", coef, ex)        # (kz, ky, nx)
        t2 = np.einsum("abx,yb->ayx", t1, ey)          # (kz, ny, nx)
        t3 = np.einsum("ayx,za->zyx", t2, ez)          # (nz, ny, nx)
        return t3.real
    import torch
    dev = torch.device(torch_device)
    C = torch.as_tensor(coef, dtype=torch.complex128, device=dev)
    EX = torch.as_tensor(ex, device=dev)
    EY = torch.as_tensor(ey, device=dev)
    EZ = torch.as_tensor(ez, device=dev)
    t1 = torch.einsum("abc,xc->abx", C, EX)
    t2 = torch.einsum("abx,yb->ayx", t1, EY)
    nz = pos_z.size
    out = torch.empty((nz, pos_y.size, pos_x.size), dtype=torch.float64, device=dev)
    for z0 in range(0, nz, chunk):
        z1 = min(nz, z0 + chunk)
        out[z0:z1] = torch.einsum("ayx,za->zyx", t2, EZ[z0:z1]).real
    return out


def turbulence(n, seed_v=910285, seed_a=910286, gamma=5.0 / 3.0, mach=1.0, beta=1.0, kmax=8,
               device=None, dtype=None):
    """rho = 1, p = 1; v Gaussian random phases with |v_k|^2 ~ k^-2 on
    1 <= |k| <= 8, scaled to rms Mach ``mach``; b = curl of an edge vector
    potential with the same spectrum (discretely divergence-free), scaled to
    plasma beta ``beta`` (b_rms^2 = 2 p / beta).  No mean field.

    With ``device`` (a torch device string) the state is built there and a
    torch tensor of shape (8, n, n, n) and dtype ``dtype`` (default float64) is
    returned inside the Workload instead of a numpy array."""
    cv = turbulence_coefficients(seed_v, kmax)
    ca = turbulence_coefficients(seed_a, kmax)
    h = 1.0 / n
    cen = (np.arange(n) + 0.5) * h
    fac = (np.arange(n) + 1.0) * h
    if device is None:
        xp_abs = np.abs
        v = [_synth(cv[c], cen, cen, cen, kmax) for c in range(3)]
        Ax = _synth(ca[0], cen, fac, fac, kmax)
        Ay = _synth(ca[1], fac, cen, fac, kmax)
        Az = _synth(ca[2], fac, fac, cen, kmax)
        roll = np.roll
        sqrt = np.sqrt
    else:
        import torch
        v = [_synth(cv[c], cen, cen, cen, kmax, device) for c in range(3)]
        Ax = _synth(ca[0], cen, fac, fac, kmax, device)
        Ay = _synth(ca[1], fac, cen, fac, kmax, device)
        Az = _synth(ca[2], fac, fac, cen, kmax, device)
        roll = lambda a, s, axis: torch.roll(a, s, dims=axis)  # noqa: E731
        sqrt = torch.sqrt

    def dm(a, axis):
        return a - roll(a, 1, axis=axis)

    bx = dm(Az, 1) / h - dm(Ay, 0) / h
    by = dm(Ax, 0) / h - dm(Az, 2) / h
    bz = dm(Ay, 2) / h - dm(Ax, 1) / h
    cs = math.sqrt(gamma * 1.0 / 1.0)
    vrms = sqrt((v[0] ** 2 + v[1] ** 2 + v[2] ** 2).mean())
    vs = mach * cs / float(vrms)
    v = [c * vs for c in v]
    brms = sqrt((bx ** 2 + by ** 2 + bz ** 2).mean())
    bs = math.sqrt(2.0 * 1.0 / beta) / float(brms)
    bx, by, bz = bx * bs, by * bs, bz * bs
    if device is None:
        st = assemble(np.ones((n, n, n)), tuple(v), 1.0, (bx, by, bz), gamma, BC_PERIODIC)
    else:
        import torch
        dt_ = torch.float64 if dtype is None else dtype
        st = torch.empty((8, n, n, n), dtype=dt_, device=device)
        # b_c (periodic): mean of faces c-1/2 and c+1/2
        bcx = 0.5 * (roll(bx, 1, 2) + bx)
        bcy = 0.5 * (roll(by, 1, 1) + by)
        bcz = 0.5 * (roll(bz, 1, 0) + bz)
        E = 1.0 / (gamma - 1.0) + 0.5 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) \
            + 0.5 * (bcx ** 2 + bcy ** 2 + bcz ** 2)
        st[0] = 1.0
        st[1], st[2], st[3] = v[0], v[1], v[2]
        st[4] = E
        st[5], st[6], st[7] = bx, by, bz
    return Workload("turbulence", st, gamma, (h, h, h), BC_PERIODIC,
                    meta={"seed_v": seed_v, "seed_a": seed_a, "mach": mach, "beta": beta})


# --------------------------------------------------------------------------
# batch of uneven boxes
# --------------------------------------------------------------------------

BATCH_SIZES = tuple(range(32, 161, 16))


def batch_specs(nbox=64, seed=2009, sizes=BATCH_SIZES):
    """Seeded list of (kind, (nx, ny, nz), axis) for the uneven batch: sizes
    drawn independently per axis, kinds round-robin Sod / Brio-Wu / blast,
    tube axis random."""
    rng = np.random.RandomState(seed)
    kinds = ("sod", "brio_wu", "blast")
    out = []
    for b in range(nbox):
        dims = tuple(int(s) for s in rng.choice(sizes, size=3))
        axis = int(rng.randint(0, 3))
        out.append((kinds[b % 3], dims, axis))
    return out


def batch_box(kind, dims, axis):
    """Initial state of one batch box (tube along ``axis`` uses the box's
    extent along that axis; transverse extents as drawn)."""
    nx, ny, nz = dims
    if kind in ("sod", "brio_wu"):
        n = dims[axis]
        if kind == "sod":
            w = shock_tube(n, axis, 1)
        else:
            w = shock_tube(n, axis, 1, gamma=2.0, b_n=0.75, b_t=(1.0, -1.0), name="brio_wu")
        # replicate the 1-D profile over the transverse extents
        reps = [nz, ny, nx]
        reps[2 - axis] = 1
        st = np.tile(w.state, [1] + reps)
        h = [1.0 / nx, 1.0 / ny, 1.0 / nz]
        return Workload(kind, np.ascontiguousarray(st), w.gamma, tuple(h), BC_OUTFLOW,
                        meta={"axis": axis})
    return blast(nx, ny, nz)


# --------------------------------------------------------------------------
# the paper's other validation problems (Sec. 4): cell-centre sampling of the
# printed initial conditions, uniform fields given on the faces
# --------------------------------------------------------------------------

def _cube(n, L=1.0):
    xc, _, _, h = _grid(n, L)
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    return X, Y, Z, h


SEDOV_T_END = 1.7419e-4
SEDOV_E_TOTAL = 3.0e5


def sedov(n=256, E_total=SEDOV_E_TOTAL, e_out=1e-3, r_in=0.01, gamma=5.0 / 3.0):
    """Sedov-Taylor blast on [0,1]^3 (Sec. 4, Sedov-Taylor blast wave): rho =
    1, v = 0, b = 0, the energy E_total spread uniformly over the cells whose
    centre lies within r_in of the box centre, specific internal energy
    e_out elsewhere; outflow boundaries.  The printed e = 3e3 inside r < 0.01
    is not consistent with the printed end state (shock at r ~ 0.45 at
    t = 1.7419e-4); E_total = 3e5 is (reading of the garbled value)."""
    X, Y, Z, h = _cube(n)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    inside = r < max(r_in, 0.5 * math.sqrt(3.0) * h * 1.0001)  # at least the central cells
    ncell = int(inside.sum())
    e_in = E_total / (ncell * h ** 3)  # energy per volume, rho = 1
    p = np.where(inside, (gamma - 1.0) * e_in, (gamma - 1.0) * e_out)
    one = np.ones(X.shape)
    z = 0 * one
    st = assemble(one, (z, z, z), p, (z, z, z), gamma, BC_OUTFLOW)
    return Workload("sedov", st, gamma, (h, h, h), BC_OUTFLOW,
                    meta={"t_end": SEDOV_T_END, "E": E_total, "cells_inside": ncell})


def spherical_riemann(n=256, gamma=5.0 / 3.0, R=0.25):
    """Spherical Sod problem on [0,1]^3 (Sec. 4, spherical Riemann problem):
    rho = 0.125, p = 0.1 inside r < 0.25 of the centre, rho = 1, p = 1
    outside, v = 0, b = 0; run to t = 0.09; outflow boundaries."""
    X, Y, Z, h = _cube(n)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    rho = np.where(r < R, 0.125, 1.0)
    p = np.where(r < R, 0.1, 1.0)
    z = 0 * rho
    st = assemble(rho, (z, z, z), p, (z, z, z), gamma, BC_OUTFLOW)
    return Workload("spherical_riemann", st, gamma, (h, h, h), BC_OUTFLOW, meta={"t_end": 0.09})


MAGNETIC_EXPLOSION_RANGES = {  # printed ranges at t = 0.03 (Sec. 4, magnetic explosion, 256^3)
    "rho": (0.24, 2.17), "p": (0.25, 15.85), "e_mag": (7.66, 33.50), "e_kin": (0.0, 17.33)}


def magnetic_explosion(n=256, gamma=5.0 / 3.0):
    """Magnetic explosion on [0,1]^3 (Sec. 4): rho = 1, v = 0, p = 100 for
    r < 0.1, p = 1 for r > 0.125, linear in r between; b = (7, 7, 0)/sqrt(2);
    run to t = 0.03 with CFL 0.5 and the minmod limiter; outflow boundaries."""
    X, Y, Z, h = _cube(n)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    p = np.where(r < 0.1, 100.0, np.where(r > 0.125, 1.0, 100.0 + (1.0 - 100.0) * (r - 0.1) / 0.025))
    one = np.ones(X.shape)
    b0 = 7.0 / math.sqrt(2.0)
    st = assemble(one, (0 * one,) * 3, p, (b0 * one, b0 * one, 0 * one), gamma, BC_OUTFLOW)
    return Workload("magnetic_explosion", st, gamma, (h, h, h), BC_OUTFLOW,
                    meta={"t_end": 0.03, "cfl": 0.5, "limiter": "minmod", "ranges": MAGNETIC_EXPLOSION_RANGES})


def rotor(n=256, gamma=1.4, r0=0.1, r1=0.115):
    """First rotor problem (Sec. 4, the rotor problem) on [0,1]^2 x one
    cell: rho = 10 and rigid rotation v = 2 (-(y-1/2), x-1/2)/r0 for r < r0,
    the tapered profile f = (r1-r)/(r1-r0) for r0 < r < r1, rho = 1 at rest
    beyond; p = 1, b = (5/sqrt(4 pi), 0, 0); run to t = 0.15; outflow
    boundaries (none are printed: reading)."""
    xc, _, _, h = _grid(n)
    Y, X = np.meshgrid(xc, xc, indexing="ij")
    dx, dy = X - 0.5, Y - 0.5
    r = np.sqrt(dx * dx + dy * dy)
    f = np.clip((r1 - r) / (r1 - r0), 0.0, 1.0)
    rho = np.where(r < r0, 10.0, np.where(r < r1, 1.0 + 9.0 * f, 1.0))
    rs = np.maximum(r, 1e-300)
    vx = np.where(r < r0, -2.0 * dy / r0, np.where(r < r1, -2.0 * f * dy / rs, 0.0))
    vy = np.where(r < r0, 2.0 * dx / r0, np.where(r < r1, 2.0 * f * dx / rs, 0.0))
    rho, vx, vy = rho[None], vx[None], vy[None]
    one = np.ones(rho.shape)
    st = assemble(rho, (vx, vy, 0 * one), 1.0, (5.0 / math.sqrt(4.0 * math.pi) * one, 0 * one, 0 * one),
                  gamma, BC_OUTFLOW)
    return Workload("rotor", st, gamma, (h, h, h), BC_OUTFLOW, meta={"t_end": 0.15})


MHD_RIEMANN_2D_RANGES = {  # printed ranges at t = 0.8 (Sec. 4, two-dimensional MHD Riemann problem, 512^2)
    "rho": (0.3428, 2.5698), "p": (0.1208, 0.7757), "e_mag": (0.0039, 0.2953), "e_kin": (0.0, 0.6233)}


def mhd_riemann_2d(n=512, L=0.8, gamma=5.0 / 3.0):
    """Two-dimensional MHD Riemann problem (Sec. 4) on [0,0.8]^2 x one cell:
    four quadrant states (rho, v_x, v_y, v_z, p) as printed, uniform
    b = (2, 0, 1)/sqrt(4 pi); zeroth-order extrapolation boundaries; run to
    t = 0.8."""
    xc, _, _, h = _grid(n, L)
    Y, X = np.meshgrid(xc, xc, indexing="ij")
    left, low = X <= L / 2, Y <= L / 2
    rho = np.where(low, np.where(left, 1.0, 3.0), np.where(left, 2.0, 1.0))
    vx = np.where(low, -0.75, 0.75)
    vy = np.where(left, 0.5, -0.5)
    rho, vx, vy = rho[None], vx[None], vy[None]
    one = np.ones(rho.shape)
    s = 1.0 / math.sqrt(4.0 * math.pi)
    st = assemble(rho, (vx, vy, 0 * one), 1.0, (2.0 * s * one, 0 * one, s * one), gamma, BC_OUTFLOW)
    return Workload("mhd_riemann_2d", st, gamma, (h, h, h), BC_OUTFLOW,
                    meta={"t_end": 0.8, "ranges": MHD_RIEMANN_2D_RANGES})
