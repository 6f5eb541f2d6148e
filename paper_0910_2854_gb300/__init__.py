"""Python binding of libfish.so, the GB300 implementation of FISH's
operator-split ideal-MHD sweep (Kaeppeli et al., arXiv:0910.2854).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``csrc/`` behind the C ABI declared in ``include/fish.h``.  The
functions below carry the C names; :class:`Box` wraps them for convenience.
PyTorch provides device memory (its caching allocator is installed as the
library's allocator) and streams.  There is no CPU fallback: if the CUDA
library is missing or no GPU is present, calls raise :class:`FishError`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfish.so")

FISH_OK, FISH_ERR_ARG, FISH_ERR_CUDA, FISH_ERR_OOM, FISH_ERR_STATE, FISH_ERR_NONPHYSICAL, FISH_ERR_TIMEOUT = range(7)
FISH_BC_PERIODIC, FISH_BC_OUTFLOW = 0, 1
(FISH_OPT_PRECISION, FISH_OPT_LIMITER, FISH_OPT_HSE, FISH_OPT_PRED_DISS, FISH_OPT_DX, FISH_OPT_DY, FISH_OPT_DZ,
 FISH_OPT_GRAVITY, FISH_OPT_KERNELS) = range(9)
FISH_KERNELS_COLUMN, FISH_KERNELS_RING = 0, 1
FISH_PREC_FP64, FISH_PREC_FP32 = 0, 1
FISH_LIM_VANLEER, FISH_LIM_MINMOD, FISH_LIM_NONE, FISH_LIM_HYBRID = 0, 1, 2, 3
FISH_GRAV_UNSPLIT, FISH_GRAV_SPLIT = 0, 1
FISH_F64, FISH_F32 = 0, 1
FISH_OP_FLUID, FISH_OP_CT = 0, 1
FISH_BATCH_OPT_LIMITER, FISH_BATCH_OPT_ORDER, FISH_BATCH_OPT_GROUPS, FISH_BATCH_OPT_GRID, FISH_BATCH_OPT_CTROWS = range(5)

# every symbol include/fish.h declares (checked by the CPU test suite)
EXPORTS = ("fish_create", "fish_set_option", "fish_set_stream", "fish_set_allocator", "fish_set_state",
           "fish_set_state_device", "fish_set_state_host", "fish_set_potential", "fish_set_mesh", "fish_cfl_dt", "fish_step", "fish_step_cfl",
           "fish_last_dt", "fish_apply", "fish_get_state", "fish_get_state_host", "fish_get_state_device", "fish_get_planes", "fish_set_planes", "fish_cfl_dt_planes", "fish_diagnostics",
           "fish_sync", "fish_clear_error", "fish_last_error", "fish_launch_count", "fish_destroy",
           "fish_diagnostics_noalloc", "fish_probe_fp64_fma", "fish_batch_create", "fish_batch_set_option", "fish_batch_set_stream",
           "fish_batch_set_state", "fish_batch_step", "fish_batch_get_state", "fish_batch_last_dt",
           "fish_batch_sync", "fish_batch_last_error", "fish_batch_launch_count", "fish_batch_cells",
           "fish_batch_destroy")

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


class FishError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


def load(path: str = LIB_PATH):
    """Load libfish.so (raises FishError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FishError(FISH_ERR_CUDA, "CUDA library %s not built (run __graft_entry__.build())" % path)
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        sig = {
            "fish_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
            "fish_set_option": ([P, ctypes.c_int, ctypes.c_double], ctypes.c_int),
            "fish_set_stream": ([P, P], ctypes.c_int),
            "fish_set_allocator": ([P, _ALLOC_T, _FREE_T, P], ctypes.c_int),
            "fish_set_state": ([P, D], ctypes.c_int),
            "fish_set_state_device": ([P, P, ctypes.c_int], ctypes.c_int),
            "fish_set_state_host": ([P, P, ctypes.c_int], ctypes.c_int),
            "fish_set_potential": ([P, D], ctypes.c_int),
            "fish_probe_fp64_fma": ([D], ctypes.c_int),
            "fish_set_mesh": ([P, D, D, D], ctypes.c_int),
            "fish_cfl_dt": ([P, ctypes.c_double, D], ctypes.c_int),
            "fish_step": ([P, ctypes.c_double], ctypes.c_int),
            "fish_step_cfl": ([P, ctypes.c_double, ctypes.c_int], ctypes.c_int),
            "fish_last_dt": ([P, D], ctypes.c_int),
            "fish_apply": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_double], ctypes.c_int),
            "fish_get_state": ([P, D], ctypes.c_int),
            "fish_get_state_device": ([P, P, ctypes.c_int], ctypes.c_int),
            "fish_get_state_host": ([P, P, ctypes.c_int], ctypes.c_int),
            "fish_get_planes": ([P, ctypes.c_int, ctypes.c_int, P], ctypes.c_int),
            "fish_cfl_dt_planes": ([P, ctypes.c_double, ctypes.c_int, ctypes.c_int, D], ctypes.c_int),
            "fish_set_planes": ([P, ctypes.c_int, ctypes.c_int, P], ctypes.c_int),
            "fish_diagnostics": ([P, D], ctypes.c_int),
            "fish_sync": ([P], ctypes.c_int),
            "fish_clear_error": ([P], ctypes.c_int),
            "fish_last_error": ([P], ctypes.c_char_p),
            "fish_launch_count": ([P], ctypes.c_longlong),
            "fish_destroy": ([P], None),
            "fish_diagnostics_noalloc": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P], ctypes.c_int),
            "fish_batch_create": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), D, ctypes.POINTER(ctypes.c_int), D,
                                   ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
            "fish_batch_set_option": ([P, ctypes.c_int, ctypes.c_double], ctypes.c_int),
            "fish_batch_set_stream": ([P, P], ctypes.c_int),
            "fish_batch_set_state": ([P, ctypes.c_int, D], ctypes.c_int),
            "fish_batch_step": ([P, ctypes.c_double, ctypes.c_int], ctypes.c_int),
            "fish_batch_get_state": ([P, ctypes.c_int, D], ctypes.c_int),
            "fish_batch_last_dt": ([P, D], ctypes.c_int),
            "fish_batch_sync": ([P], ctypes.c_int),
            "fish_batch_last_error": ([P], ctypes.c_char_p),
            "fish_batch_launch_count": ([P], ctypes.c_longlong),
            "fish_batch_cells": ([P], ctypes.c_longlong),
            "fish_batch_destroy": ([P], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Box:
    """One box of nx*ny*nz cells on the GPU (wraps a fish_ctx).

    State arrays have shape (8, nz, ny, nx): rho, m_x, m_y, m_z, E, b_x
    (faces i+1/2), b_y (faces j+1/2), b_z (faces k+1/2)."""

    def __init__(self, nx, ny, nz, gamma, bc=FISH_BC_PERIODIC, precision="fp64", limiter=FISH_LIM_VANLEER,
                 hse=False, pred_diss=1.0, h=None, use_torch_allocator=True, stream=None, gravity="unsplit",
                 kernels="column"):
        self._lib = load()
        self.n = (int(nx), int(ny), int(nz))
        self.precision = precision
        h_ = ctypes.c_void_p()
        self._check(self._lib.fish_create(self.n[0], self.n[1], self.n[2], float(gamma), int(bc), ctypes.byref(h_)),
                    "fish_create")
        self.ctx = h_
        self._cb = None
        self._torch_stream = None
        try:
            if precision not in ("fp64", "fp32"):
                raise ValueError("precision must be 'fp64' or 'fp32'")
            self.set_option(FISH_OPT_PRECISION, FISH_PREC_FP64 if precision == "fp64" else FISH_PREC_FP32)
            self.set_option(FISH_OPT_LIMITER, int(limiter))
            if gravity not in ("unsplit", "split"):
                raise ValueError("gravity must be 'unsplit' or 'split'")
            self.set_option(FISH_OPT_GRAVITY, FISH_GRAV_SPLIT if gravity == "split" else FISH_GRAV_UNSPLIT)
            self.set_option(FISH_OPT_HSE, 1 if hse else 0)
            self.set_option(FISH_OPT_PRED_DISS, float(pred_diss))
            if kernels not in ("column", "ring"):
                raise ValueError("kernels must be 'column' or 'ring'")
            if kernels == "ring":
                self.set_option(FISH_OPT_KERNELS, FISH_KERNELS_RING)
            if h is not None:
                for k, v in zip((FISH_OPT_DX, FISH_OPT_DY, FISH_OPT_DZ), h):
                    self.set_option(k, float(v))
            self._attach_torch(use_torch_allocator, stream)
        except Exception:
            self.close()
            raise

    # -- plumbing -----------------------------------------------------------
    def _attach_torch(self, use_alloc, stream):
        try:
            import torch
        except ImportError:
            return
        if not torch.cuda.is_available():
            return
        dev = torch.cuda.current_device()
        self._torch_stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self._check(self._lib.fish_set_stream(self.ctx, ctypes.c_void_p(self._torch_stream.cuda_stream)),
                    "fish_set_stream")
        if use_alloc:
            s = self._torch_stream

            def _alloc(size, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), device=dev, stream=s)
                except Exception:
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = (_ALLOC_T(_alloc), _FREE_T(_free))
            self._check(self._lib.fish_set_allocator(self.ctx, self._cb[0], self._cb[1], None), "fish_set_allocator")

    @property
    def stream(self):
        """The torch.cuda.Stream the library queues its work on."""
        return self._torch_stream

    def _check(self, code, what):
        if code != FISH_OK:
            msg = ""
            if getattr(self, "ctx", None):
                msg = self._lib.fish_last_error(self.ctx).decode(errors="replace")
            raise FishError(code, "%s failed: %s" % (what, msg))

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.fish_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI -------------------------------------------------------------
    def set_option(self, key, value):
        self._check(self._lib.fish_set_option(self.ctx, int(key), float(value)), "fish_set_option")

    def set_state(self, state):
        """Upload a state: numpy (host, FP64) or a torch CUDA tensor (f64/f32)."""
        if hasattr(state, "is_cuda") and state.is_cuda:
            import torch
            t = state.contiguous()
            if t.numel() != 8 * np.prod(self.n):
                raise ValueError("state has %d values, expected %d" % (t.numel(), 8 * np.prod(self.n)))
            dt = FISH_F64 if t.dtype == torch.float64 else FISH_F32
            if t.dtype not in (torch.float64, torch.float32):
                raise ValueError("device state must be float64 or float32")
            torch.cuda.current_stream().synchronize()
            self._check(self._lib.fish_set_state_device(self.ctx, ctypes.c_void_p(t.data_ptr()), dt),
                        "fish_set_state_device")
            self.sync()
            return
        a = np.ascontiguousarray(state, dtype=np.float64)
        if a.size != 8 * np.prod(self.n):
            raise ValueError("state has %d values, expected %d" % (a.size, 8 * np.prod(self.n)))
        self._check(self._lib.fish_set_state(self.ctx, _dptr(a)), "fish_set_state")

    def set_state_host(self, state):
        """Upload from a host buffer (numpy array or CPU torch tensor, ideally
        pinned), float64 or float32, without conversion on the host."""
        if hasattr(state, "data_ptr"):
            import torch
            if state.dtype not in (torch.float64, torch.float32) or not state.is_contiguous():
                raise ValueError("host state must be a contiguous float64/float32 tensor")
            ptr, dt, size = state.data_ptr(), (FISH_F64 if state.dtype == torch.float64 else FISH_F32), state.numel()
        else:
            a = np.ascontiguousarray(state)
            if a.dtype not in (np.float64, np.float32):
                a = a.astype(np.float64)
            ptr, dt, size = a.ctypes.data, (FISH_F64 if a.dtype == np.float64 else FISH_F32), a.size
            self._keep = a
        if size != 8 * np.prod(self.n):
            raise ValueError("state has %d values, expected %d" % (size, 8 * np.prod(self.n)))
        self._check(self._lib.fish_set_state_host(self.ctx, ctypes.c_void_p(ptr), dt), "fish_set_state_host")

    def set_potential(self, phi):
        if phi is None:
            self._check(self._lib.fish_set_potential(self.ctx, None), "fish_set_potential")
            return
        a = np.ascontiguousarray(phi, dtype=np.float64)
        if a.size != np.prod(self.n):
            raise ValueError("potential has the wrong size")
        self._check(self._lib.fish_set_potential(self.ctx, _dptr(a)), "fish_set_potential")

    def set_mesh(self, widths):
        """Irregular Cartesian mesh: widths = (dx, dy, dz), each None (the
        uniform width of that axis) or an array of the axis' cell widths;
        None restores the uniform mesh."""
        arrs = [None, None, None]
        if widths is not None:
            for d, wd in enumerate(widths):
                if wd is not None:
                    a = np.ascontiguousarray(wd, dtype=np.float64).reshape(-1)
                    if a.size != self.n[d]:
                        raise ValueError("widths[%d] needs %d entries" % (d, self.n[d]))
                    arrs[d] = a
        self._mesh = arrs  # keep the host arrays alive for the call
        self._check(self._lib.fish_set_mesh(self.ctx, *[None if a is None else _dptr(a) for a in arrs]),
                    "fish_set_mesh")

    def cfl_dt(self, k):
        out = ctypes.c_double()
        self._check(self._lib.fish_cfl_dt(self.ctx, float(k), ctypes.byref(out)), "fish_cfl_dt")
        return out.value

    def cfl_dt_planes(self, k, k0, nk):
        """CFL time step over the z-planes k0 .. k0+nk-1 only."""
        out = ctypes.c_double()
        self._check(self._lib.fish_cfl_dt_planes(self.ctx, float(k), int(k0), int(nk), ctypes.byref(out)),
                    "fish_cfl_dt_planes")
        return out.value

    def step(self, dt, nsteps=1):
        for _ in range(int(nsteps)):
            self._check(self._lib.fish_step(self.ctx, float(dt)), "fish_step")

    def step_cfl(self, k, nsteps=1):
        self._check(self._lib.fish_step_cfl(self.ctx, float(k), int(nsteps)), "fish_step_cfl")

    def last_dt(self):
        out = ctypes.c_double()
        self._check(self._lib.fish_last_dt(self.ctx, ctypes.byref(out)), "fish_last_dt")
        return out.value

    def apply(self, op, direction, dt):
        self._check(self._lib.fish_apply(self.ctx, int(op), int(direction), float(dt)), "fish_apply")

    def fluid(self, direction, dt):
        self.apply(FISH_OP_FLUID, direction, dt)

    def ct(self, direction, dt):
        self.apply(FISH_OP_CT, direction, dt)

    def get_state(self):
        out = np.empty((8, self.n[2], self.n[1], self.n[0]), dtype=np.float64)
        self._check(self._lib.fish_get_state(self.ctx, _dptr(out)), "fish_get_state")
        return out

    def get_state_host(self, out):
        """Download into a host buffer (contiguous CPU torch tensor, ideally
        pinned, or numpy array), float64 or float32, converted on the device."""
        if hasattr(out, "data_ptr"):
            import torch
            if out.dtype not in (torch.float64, torch.float32) or not out.is_contiguous():
                raise ValueError("host state must be a contiguous float64/float32 tensor")
            ptr, dt, size = out.data_ptr(), (FISH_F64 if out.dtype == torch.float64 else FISH_F32), out.numel()
        else:
            if out.dtype not in (np.float64, np.float32) or not out.flags.c_contiguous:
                raise ValueError("host state must be a contiguous float64/float32 array")
            ptr, dt, size = out.ctypes.data, (FISH_F64 if out.dtype == np.float64 else FISH_F32), out.size
        if size != 8 * np.prod(self.n):
            raise ValueError("state has %d values, expected %d" % (size, 8 * np.prod(self.n)))
        self._check(self._lib.fish_get_state_host(self.ctx, ctypes.c_void_p(ptr), dt), "fish_get_state_host")
        return out

    def get_planes(self, k0, nk, out):
        """z-planes k0 .. k0+nk-1 of the 8 fields into ``out`` (a contiguous
        torch tensor of 8*nk*nx*ny values of the box's precision, on the
        device or in host memory); queued on the box's stream."""
        self._check(self._lib.fish_get_planes(self.ctx, int(k0), int(nk), ctypes.c_void_p(out.data_ptr())),
                    "fish_get_planes")
        return out

    def set_planes(self, k0, nk, src):
        """The inverse of get_planes: overwrite z-planes k0 .. k0+nk-1."""
        self._check(self._lib.fish_set_planes(self.ctx, int(k0), int(nk), ctypes.c_void_p(src.data_ptr())),
                    "fish_set_planes")

    def get_state_device(self, out):
        import torch
        if out.dtype not in (torch.float64, torch.float32) or not out.is_contiguous():
            raise ValueError("output must be a contiguous float64/float32 CUDA tensor")
        if out.numel() != 8 * np.prod(self.n):
            raise ValueError("output has the wrong size")
        dt = FISH_F64 if out.dtype == torch.float64 else FISH_F32
        self._check(self._lib.fish_get_state_device(self.ctx, ctypes.c_void_p(out.data_ptr()), dt),
                    "fish_get_state_device")
        self.sync()
        return out

    def diagnostics(self):
        out = np.zeros(9, dtype=np.float64)
        self._check(self._lib.fish_diagnostics(self.ctx, _dptr(out)), "fish_diagnostics")
        return out

    def sync(self):
        self._check(self._lib.fish_sync(self.ctx), "fish_sync")

    def clear_error(self):
        self._check(self._lib.fish_clear_error(self.ctx), "fish_clear_error")

    def sync_quiet(self):
        """Wait for the queued work; a non-physical status it reported is
        returned (True) and cleared instead of raised.  Other errors raise."""
        code = self._lib.fish_sync(self.ctx)
        if code == FISH_ERR_NONPHYSICAL:
            self.clear_error()
            return True
        self._check(code, "fish_sync")
        return False

    def launch_count(self):
        return int(self._lib.fish_launch_count(self.ctx))


def diagnostics_noalloc(state, dims, bc, h, out, stream=None):
    """fish_diagnostics_noalloc: totals and max |div b| of the device state
    tensor ``state`` (float64/float32, 8*nx*ny*nz values) into the device
    tensor ``out`` (9 float64), queued on ``stream`` (a torch.cuda.Stream,
    default: the current stream).  Allocates no device memory."""
    import torch
    lib = load()
    if not (state.is_cuda and out.is_cuda and state.is_contiguous() and out.is_contiguous()):
        raise ValueError("state and out must be contiguous CUDA tensors")
    if state.dtype not in (torch.float64, torch.float32) or out.dtype != torch.float64 or out.numel() < 9:
        raise ValueError("state must be float64/float32 and out 9 float64 values")
    nx, ny, nz = (int(v) for v in dims)
    if state.numel() != 8 * nx * ny * nz:
        raise ValueError("state has the wrong size")
    s = stream if stream is not None else torch.cuda.current_stream()
    code = lib.fish_diagnostics_noalloc(ctypes.c_void_p(state.data_ptr()),
                                        FISH_F64 if state.dtype == torch.float64 else FISH_F32,
                                        nx, ny, nz, int(bc), float(h[0]), float(h[1]), float(h[2]),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if code != FISH_OK:
        raise FishError(code, "fish_diagnostics_noalloc failed")
    return out


class Batch:
    """Many independent FP32 boxes of uneven sizes advanced together (wraps
    a fish_batch).  ``dims``: list of (nx, ny, nz) (nx, ny even); ``gammas``,
    ``bcs``: per box; ``hs``: per-box cell widths or None (1/n)."""

    def __init__(self, dims, gammas, bcs, hs=None, limiter=FISH_LIM_VANLEER, stream=None):
        self._lib = load()
        self.dims = [tuple(int(v) for v in d) for d in dims]
        n = len(self.dims)
        d = (ctypes.c_int * (3 * n))(*[v for t in self.dims for v in t])
        g = (ctypes.c_double * n)(*[float(x) for x in gammas])
        b = (ctypes.c_int * n)(*[int(x) for x in bcs])
        h = None if hs is None else (ctypes.c_double * (3 * n))(*[float(v) for t in hs for v in t])
        out = ctypes.c_void_p()
        code = self._lib.fish_batch_create(n, d, g, b, h, ctypes.byref(out))
        if code != FISH_OK:
            raise FishError(code, "fish_batch_create failed")
        self.ptr = out
        self._stream = None
        try:
            self.set_option(FISH_BATCH_OPT_LIMITER, limiter)
            try:
                import torch
                if torch.cuda.is_available():
                    self._stream = stream if stream is not None else torch.cuda.Stream()
                    self._check(self._lib.fish_batch_set_stream(self.ptr, ctypes.c_void_p(self._stream.cuda_stream)),
                                "fish_batch_set_stream")
            except ImportError:
                pass
        except Exception:
            self.close()
            raise

    @property
    def stream(self):
        return self._stream

    def _check(self, code, what):
        if code != FISH_OK:
            msg = self._lib.fish_batch_last_error(self.ptr).decode(errors="replace") if self.ptr else ""
            raise FishError(code, "%s failed: %s" % (what, msg))

    def set_option(self, key, value):
        self._check(self._lib.fish_batch_set_option(self.ptr, int(key), float(value)), "fish_batch_set_option")

    def set_state(self, box, state):
        a = np.ascontiguousarray(state, dtype=np.float64)
        if a.size != 8 * int(np.prod(self.dims[box])):
            raise ValueError("state of box %d has the wrong size" % box)
        self._check(self._lib.fish_batch_set_state(self.ptr, int(box), _dptr(a)), "fish_batch_set_state")

    def step(self, k, nsteps=1):
        self._check(self._lib.fish_batch_step(self.ptr, float(k), int(nsteps)), "fish_batch_step")

    def get_state(self, box):
        nx, ny, nz = self.dims[box]
        out = np.empty((8, nz, ny, nx), dtype=np.float64)
        self._check(self._lib.fish_batch_get_state(self.ptr, int(box), _dptr(out)), "fish_batch_get_state")
        return out

    def last_dt(self):
        out = np.zeros(len(self.dims), dtype=np.float64)
        self._check(self._lib.fish_batch_last_dt(self.ptr, _dptr(out)), "fish_batch_last_dt")
        return out

    def sync(self):
        self._check(self._lib.fish_batch_sync(self.ptr), "fish_batch_sync")

    @property
    def cells(self):
        return int(self._lib.fish_batch_cells(self.ptr))

    def launch_count(self):
        return int(self._lib.fish_batch_launch_count(self.ptr))

    def close(self):
        if getattr(self, "ptr", None):
            self._lib.fish_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_fp64_fma():
    """FP64 fused multiply-adds per second of the current device (the peak
    the FP64 sweeps are compared against)."""
    lib = load()
    out = ctypes.c_double()
    code = lib.fish_probe_fp64_fma(ctypes.byref(out))
    if code != FISH_OK:
        raise FishError(code, "fish_probe_fp64_fma failed")
    return out.value
