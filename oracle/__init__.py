"""FP64 CPU oracle of FISH's operator-split MHD step (arXiv:0910.2854).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  It
shares no code with the CUDA path in ``paper_0910_2854_gb300/`` and never
imports it.

The numerics live in ``fish_oracle.c`` (plain C, IEEE double, compiled with
``-ffp-contract=off``); this module only builds that file with gcc and
marshals numpy arrays through ctypes.

Parity status of the functions (what pins each one; see ``tests/test_oracle_*``):
  * ``OracleBox.step`` / ``fluid`` / ``ct``: pinned by the exact Sod Riemann
    solution, the circularly polarised Alfven wave after one period,
    second-order convergence on smooth advection, conservation and
    div b = 0 to round-off, axis-permutation symmetry and the limiter-off
    reduction to the textbook Rusanov predictor-corrector; the constrained
    transport's upwind predictor and face-velocity smoothing (eq0362-eq0364)
    by closed forms of the linearised operator: the amplification factor of
    a single field mode in a uniform flow and the cos^2(theta/2) transfer
    function of the smoothing in the response to a velocity mode.
  * hydrostatic-gradient correction (``hse=True``): pinned by a discrete
    hydrostatic atmosphere, in which the corrected acoustic dissipation of
    the mass flux vanishes; the polytrope behaviour of the paper's Sec. 4 is
    not yet reproduced, so its second-order construction is partly unpinned.
  * ``cfl``: pinned by closed-form fast speeds on a uniform state.
  * hybrid limiter (``limiter=LIM_HYBRID``): pinned by its two limits (a
    subsonic flow gives the Van Leer result bitwise, a supersonic one the
    minmod result) and a mixed flow that differs from both.
  * operator-split gravity (``gravity_split=True``): pinned by the exact
    impulse and kinetic-energy change of a uniform state in a linear
    potential.
  * irregular Cartesian meshes (``widths=``): pinned by equal widths giving
    the uniform method to round-off, conservation of the volume-weighted
    totals and of the per-cell-width divergence, a uniform state staying
    uniform, exact free fall in a linear potential (split and unsplit), the
    commutation with a reflection of state and mesh, exact shear-flow face
    velocities, the closed-form CFL step and, for the edge-velocity weights
    along the sweep, the upwind choice at an interface where the linearly
    interpolated velocity changes sign.
  * ``test_oracle_mutants.py`` plants mistakes in a copy of the source and
    checks that the pins catch each of them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fish_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfish_oracle.so")

LIM_VANLEER, LIM_MINMOD, LIM_NONE, LIM_HYBRID = 0, 1, 2, 3
BC_PERIODIC, BC_OUTFLOW = 0, 1
FIELDS = ("rho", "mx", "my", "mz", "E", "bx", "by", "bz")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fish_oracle.c into a shared library with gcc (no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def build_variant(source_text: str, tag: str) -> str:
    """Compile a modified copy of the oracle source (used by the mutation test,
    which plants mistakes in the oracle to show that the pins catch them)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, "variant_%s.c" % tag)
    lib = os.path.join(_BUILD, "libvariant_%s.so" % tag)
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-fno-fast-math", "-o", lib, src, "-lm"], check=True)
    return lib


def source() -> str:
    with open(_SRC) as f:
        return f.read()


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("bc", ctypes.c_int),
                ("limiter", ctypes.c_int), ("hse", ctypes.c_int),
                ("pred_diss", ctypes.c_double),
                ("phi", ctypes.POINTER(ctypes.c_double)),
                ("gravity_split", ctypes.c_int),
                ("w", ctypes.POINTER(ctypes.c_double) * 3)]


def _bind(lib):
    P = ctypes.POINTER(_Problem)
    D = ctypes.POINTER(ctypes.c_double)
    lib.oracle_fluid.argtypes = [P, D, ctypes.c_int, ctypes.c_double]
    lib.oracle_fluid.restype = ctypes.c_int
    lib.oracle_ct.argtypes = [P, D, ctypes.c_int, ctypes.c_double]
    lib.oracle_ct.restype = ctypes.c_int
    lib.oracle_step.argtypes = [P, D, ctypes.c_double, ctypes.c_int]
    lib.oracle_step.restype = ctypes.c_int
    lib.oracle_cfl.argtypes = [P, D, ctypes.c_double]
    lib.oracle_cfl.restype = ctypes.c_double
    lib.oracle_cfl_planes.argtypes = [P, D, ctypes.c_double, ctypes.c_long, ctypes.c_long]
    lib.oracle_cfl_planes.restype = ctypes.c_double
    lib.oracle_diag.argtypes = [P, D, D]
    lib.oracle_diag.restype = None
    return lib


def load_library(path):
    """ctypes handle of an oracle build at ``path`` (see build_variant)."""
    return _bind(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class OracleError(RuntimeError):
    pass


class OracleBox:
    """One box of nx*ny*nz cells advanced by the CPU oracle.

    ``state`` is a float64 array of shape (8, nz, ny, nx) (x fastest):
    rho, m_x, m_y, m_z, E, b_x (face i+1/2), b_y (face j+1/2), b_z (face k+1/2).
    """

    def __init__(self, nx, ny, nz, gamma, bc=BC_PERIODIC, h=None,
                 limiter=LIM_VANLEER, hse=False, pred_diss=1.0, phi=None, gravity_split=False, widths=None,
                 lib=None):
        self._lib = lib
        self.n = (int(nx), int(ny), int(nz))
        if h is None:
            h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
        self.h = tuple(float(v) for v in h)
        self.gamma = float(gamma)
        self.bc = int(bc)
        self.limiter = int(limiter)
        self.hse = bool(hse)
        self.pred_diss = float(pred_diss)
        self.gravity_split = bool(gravity_split)
        self.state = np.zeros((8, nz, ny, nx), dtype=np.float64)
        self.phi = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64).reshape(nz, ny, nx)
        # irregular Cartesian mesh (eq037): per axis None (uniform h) or the cell widths
        self.widths = [None, None, None]
        if widths is not None:
            for d, wd in enumerate(widths):
                if wd is not None:
                    wd = np.ascontiguousarray(wd, dtype=np.float64).reshape(-1)
                    if wd.size != self.n[d] or not np.all(wd > 0):
                        raise ValueError("widths[%d] needs %d positive entries" % (d, self.n[d]))
                    self.widths[d] = wd
        self.flags = 0

    # -- marshalling -------------------------------------------------------
    def _L(self):
        return self._lib if self._lib is not None else _load()

    def _problem(self):
        p = _Problem()
        p.n[:] = self.n
        p.h[:] = self.h
        p.gamma = self.gamma
        p.bc = self.bc
        p.limiter = self.limiter
        p.hse = 1 if self.hse else 0
        p.pred_diss = self.pred_diss
        p.gravity_split = 1 if self.gravity_split else 0
        if self.phi is not None:
            p.phi = self.phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        else:
            p.phi = ctypes.POINTER(ctypes.c_double)()
        for d in range(3):
            wd = self.widths[d]
            p.w[d] = (wd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if wd is not None
                      else ctypes.POINTER(ctypes.c_double)())
        return p

    def _ptr(self):
        if not self.state.flags["C_CONTIGUOUS"] or self.state.dtype != np.float64:
            self.state = np.ascontiguousarray(self.state, dtype=np.float64)
        return self.state.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def set_state(self, state):
        s = np.asarray(state, dtype=np.float64).reshape(8, self.n[2], self.n[1], self.n[0])
        self.state = np.ascontiguousarray(s).copy()

    # -- operators ---------------------------------------------------------
    def fluid(self, d, dt):
        """L_d(dt) (fluid sweep along axis d = 0, 1, 2)."""
        p = self._problem()
        r = self._L().oracle_fluid(ctypes.byref(p), self._ptr(), int(d), float(dt))
        if r < 0:
            raise OracleError("oracle_fluid: allocation failure")
        self.flags |= r
        return r

    def ct(self, d, dt):
        """B_d(dt) (constrained-transport sweep along axis d)."""
        p = self._problem()
        r = self._L().oracle_ct(ctypes.byref(p), self._ptr(), int(d), float(dt))
        if r < 0:
            raise OracleError("oracle_ct: allocation failure")
        return r

    def step(self, dt, nsteps=1):
        """``nsteps`` full xyzzyx double steps; each advances time by 2*dt."""
        p = self._problem()
        r = self._L().oracle_step(ctypes.byref(p), self._ptr(), float(dt), int(nsteps))
        if r < 0:
            raise OracleError("oracle_step: allocation failure")
        self.flags |= r
        return r

    def cfl(self, k):
        p = self._problem()
        return float(self._L().oracle_cfl(ctypes.byref(p), self._ptr(), float(k)))

    def cfl_planes(self, k, k0, nk):
        """The CFL step with the minimum over the z-planes k0 .. k0+nk-1."""
        p = self._problem()
        return float(self._L().oracle_cfl_planes(ctypes.byref(p), self._ptr(), float(k), int(k0), int(nk)))

    def diag(self):
        """8 volume-weighted field totals and max |div b|."""
        p = self._problem()
        out = np.zeros(9, dtype=np.float64)
        self._L().oracle_diag(ctypes.byref(p), self._ptr(),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def pressure(self):
        """Gas pressure per cell (eq0050) with the cell-centred field."""
        rho, mx, my, mz, E, bx, by, bz = self.state
        bc = self.cell_centred_b()
        kin = 0.5 * (mx * mx + my * my + mz * mz) / rho
        mag = 0.5 * (bc[0] ** 2 + bc[1] ** 2 + bc[2] ** 2)
        return (self.gamma - 1.0) * (E - kin - mag)

    def cell_centred_b(self):
        out = []
        for ax, f in enumerate((5, 6, 7)):
            b = self.state[f]
            axis = 2 - ax  # numpy axis of x, y, z in (nz, ny, nx)
            if self.bc == BC_PERIODIC:
                lo = np.roll(b, 1, axis=axis)
            else:
                idx = [slice(None)] * 3
                n = b.shape[axis]
                sel = np.concatenate([[0], np.arange(n - 1)])
                idx[axis] = sel
                lo = b[tuple(idx)]
            out.append(0.5 * (lo + b))
        return out
