"""Measurements of the GPU path beyond the throughput line of bench.py, run
on one GPU and printed as one JSON line each:

  python -m paper_0910_2854_gb300.reports polytrope [n] [tau_units]
      n = 1 polytrope (n^3, FP32 with the hydrostatic island) with and
      without the hydrostatic-gradient correction for tau_units hydrostatic
      times (default 20, as in the paper): time series of the central
      density and of the largest spurious speed inside the star.
  python -m paper_0910_2854_gb300.reports fp32_vs_fp64 [n] [steps]
      random-phase turbulence n^3: FP32 and FP64 paths each advanced with
      their own CFL steps; L1 density difference relative to the FP64 path,
      and both throughputs.
  python -m paper_0910_2854_gb300.reports batch
      the seeded batch of 64 uneven boxes: autotuned choice and throughput.
  python -m paper_0910_2854_gb300.reports variants [n] [steps]
      the FP32 turbulence box n^3 advanced with each variant of the method
      (Van Leer, hybrid limiter, irregular mesh, unsplit and split gravity
      in a smooth potential): ms per double step and cell-updates/s.
  python -m paper_0910_2854_gb300.reports fp64_sweeps [n]
      the FP64 path on the Orszag-Tang box n^3: one double step and each
      operator timed with CUDA events, next to the probed FP64 FMA rate of
      the device.
  python -m paper_0910_2854_gb300.reports validation <name> [n] [fp32|fp64] [cfl]
      one of the paper's validation problems (sedov, spherical_riemann,
      magnetic_explosion, rotor, mhd_riemann_2d) at the paper's size (or n)
      run to the paper's end time: value ranges against the printed ones,
      and for the Sedov blast the shock radius against the self-similar
      t^(2/5) law and the printed radius.

Every step runs in the CUDA kernels behind the C ABI; the inputs are the
seeded synthetic fields of ``workloads``.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import Batch, Box, autotune
from . import workloads as W


def _timed_steps(box, torch, k, steps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(box.stream)
    box.step_cfl(k, steps)
    e1.record(box.stream)
    e1.synchronize()
    box.sync()
    return e0.elapsed_time(e1)


def polytrope(n=384, tau_units=20.0, k=0.5, samples=40):
    """The n = 1 polytrope in its fixed potential (FP32, unsplit gravity),
    with and without the hydrostatic-gradient correction, for tau_units
    hydrostatic times tau_HSE = (rho_mean G)^(-1/2) / 2 (the paper's Sec. 4
    runs 20).  Records, about ``samples`` times, the central density (mean
    of the 8 cells around the centre of an even box, else the central cell)
    normalised to its initial value and the largest speed inside the star."""
    import torch
    w = W.polytrope(n)
    R, rho_c, G = 1.0, 1.0, 1.0
    M = 4.0 * R ** 3 * rho_c / math.pi
    rho_mean = M / (4.0 / 3.0 * math.pi * R ** 3)
    tau = 0.5 / math.sqrt(rho_mean * G)
    t_end = tau_units * tau
    c = n // 2
    sl = slice(c - 1, c + 1) if n % 2 == 0 else slice(c, c + 1)

    def central(st):
        return float(st[0, sl, sl, sl].mean())

    out = {"report": "polytrope", "n": n, "cfl": k, "precision": "fp32", "tau_hse": tau, "t_end": t_end,
           "rho_c0": central(w.state)}
    inside = w.state[0] > 10 * w.state[0].min()
    for hse in (False, True):
        box = Box(*w.dims, w.gamma, bc=w.bc, precision="fp32", h=w.h, hse=hse)
        box.set_state(w.state)
        box.set_potential(w.phi)
        t, steps, ms = 0.0, 0, 0.0
        series = [(0.0, 1.0, 0.0)]
        next_sample = t_end / samples
        while t < t_end:
            ms += _timed_steps(box, torch, k, 1)
            t += 2.0 * box.last_dt()
            steps += 1
            if t >= next_sample or t >= t_end:
                st = box.get_state()
                v = np.sqrt(st[1] ** 2 + st[2] ** 2 + st[3] ** 2) / st[0]
                series.append((t / tau, central(st) / out["rho_c0"], float(v[inside].max())))
                next_sample += t_end / samples
        key = "hse" if hse else "no_hse"
        out[key] = {"double_steps": steps, "ms_per_step": ms / steps,
                    "rho_c_drift_end": series[-1][1] - 1.0, "vmax_star_end": series[-1][2],
                    "series_t_over_tau_rho_c_vmax": series}
        box.close()
        torch.cuda.empty_cache()
    return out


def fp32_vs_fp64(n=1024, steps=20, k=0.5):
    import torch
    out = {"report": "fp32_vs_fp64", "n": n, "steps": steps, "cfl": k}
    rho = {}
    for prec in ("fp32", "fp64"):
        dt_ = torch.float32 if prec == "fp32" else torch.float64
        w = W.turbulence(n, device="cuda", dtype=dt_)
        box = Box(n, n, n, w.gamma, precision=prec, h=w.h)
        box.set_state(w.state)
        del w
        torch.cuda.empty_cache()
        box.step_cfl(k, 1)
        box.sync()
        ms = _timed_steps(box, torch, k, steps - 1)
        st = torch.empty(8 * n ** 3, dtype=dt_, device="cuda")
        box.get_state_device(st)
        rho[prec] = st[: n ** 3].double().cpu()
        out[prec] = {"ms_per_step": ms / (steps - 1), "cell_updates_per_s": n ** 3 / (ms / (steps - 1) * 1e-3),
                     "last_dt": box.last_dt()}
        del st
        box.close()
        torch.cuda.empty_cache()
    d = (rho["fp32"] - rho["fp64"]).abs().mean().item() / rho["fp64"].abs().mean().item()
    out["l1_rho_rel"] = d
    out["fp32_over_fp64"] = out["fp32"]["cell_updates_per_s"] / out["fp64"]["cell_updates_per_s"]
    return out


def fp64_sweeps(n=128, steps=3, k=0.5):
    import torch
    from . import FISH_OP_CT, FISH_OP_FLUID, probe_fp64_fma
    w = W.orszag_tang(n)
    box = Box(n, n, n, w.gamma, precision="fp64", h=w.h)
    box.set_state(w.state)
    box.step_cfl(k, 1)
    box.sync()
    ms = _timed_steps(box, torch, k, steps)
    dt = box.cfl_dt(k)
    out = {"report": "fp64_sweeps", "n": n, "ms_per_step": ms / steps}
    for kind, op in (("fluid", FISH_OP_FLUID), ("ct", FISH_OP_CT)):
        for d in range(3):
            box.apply(op, d, dt)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(box.stream)
            for _ in range(2):
                box.apply(op, d, dt)
            e1.record(box.stream)
            e1.synchronize()
            out["%s_%s_ms" % (kind, "xyz"[d])] = e0.elapsed_time(e1) / 2
    box.sync()
    box.close()
    out["fp64_fma_per_s"] = probe_fp64_fma()
    return out


def variants(n=512, steps=5, k=0.5):
    import torch
    from . import FISH_LIM_HYBRID
    w = W.turbulence(n, device="cuda", dtype=torch.float32)
    x = (np.arange(n) + 0.5) / n
    widths = [(1.0 + 0.3 * np.sin(2 * np.pi * (x + 0.1 * a))) / n for a in range(3)]
    widths = [wd / wd.sum() for wd in widths]
    phi = None
    out = {"report": "variants", "n": n, "steps": steps, "cfl": k, "precision": "fp32", "cases": {}}
    cases = [("vanleer", {}), ("hybrid", {"limiter": FISH_LIM_HYBRID}), ("irregular_mesh", {"mesh": True}),
             ("gravity_unsplit", {"grav": True}), ("gravity_split", {"grav": True, "gravity": "split"})]
    for name, opt in cases:
        kw = {key: opt[key] for key in ("limiter", "gravity") if key in opt}
        box = Box(n, n, n, w.gamma, precision="fp32", h=w.h, **kw)
        if opt.get("mesh"):
            box.set_mesh(widths)
        box.set_state(w.state)
        if opt.get("grav"):
            if phi is None:
                # a smooth periodic potential well, weak against the
                # turbulent pressure (|grad phi| ~ 0.5)
                zz = np.cos(2 * np.pi * x)[:, None, None]
                yy = np.cos(2 * np.pi * x)[None, :, None]
                xx = np.cos(2 * np.pi * x)[None, None, :]
                phi = -0.08 * (xx + yy + zz)
                phi = np.broadcast_to(phi, (n, n, n)).copy()
            box.set_potential(phi)
        box.step_cfl(k, 1)
        box.sync()
        ms = _timed_steps(box, torch, k, steps) / steps
        out["cases"][name] = {"ms_per_step": ms, "cell_updates_per_s": n ** 3 / (ms * 1e-3)}
        box.close()
        torch.cuda.empty_cache()
    return out


def batch(k=0.5, steps=10):
    import torch
    specs = W.batch_specs()
    ws = [W.batch_box(*s) for s in specs]
    dims = [w.dims for w in ws]
    gam = [w.gamma for w in ws]
    bcs = [w.bc for w in ws]
    hs = [w.h for w in ws]
    choice = autotune.tune(dims, gam, bcs, [w.state for w in ws], hs=hs)
    b = Batch(dims, gam, bcs, hs)
    autotune.apply(b, choice)
    for i, w in enumerate(ws):
        b.set_state(i, w.state)
    b.step(k, 3)
    b.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(k, steps)
    e1.record(b.stream)
    e1.synchronize()
    b.sync()
    ms = e0.elapsed_time(e1) / steps
    out = {"report": "batch", "boxes": len(ws), "cells": b.cells, "ms_per_step": ms,
           "cell_updates_per_s": b.cells / (ms * 1e-3), "launches_per_step": 15,
           "tuning": dict({kk: choice[kk] for kk in ("order", "groups", "grid")}, ctrows=choice.get("ctrows", 4))}
    b.close()
    return out


VALIDATION = {  # name: (generator, paper size, CFL number, limiter)
    "sedov": (W.sedov, 256, 0.5, "vanleer"),
    "spherical_riemann": (W.spherical_riemann, 256, 0.5, "vanleer"),
    "magnetic_explosion": (W.magnetic_explosion, 256, 0.5, "minmod"),
    "rotor": (W.rotor, 256, 0.5, "vanleer"),
    "mhd_riemann_2d": (W.mhd_riemann_2d, 512, 0.5, "vanleer"),
}


class StoppedEarly(Exception):
    """The run met a non-physical state before the end time."""

    def __init__(self, t, steps, msg):
        super().__init__(msg)
        self.t, self.steps = t, steps


def run_to(box, t_end, k, t=0.0, max_steps=200000):
    """Double steps with the CFL time step of the current state, the last
    one shortened to land on t_end; returns (t, double steps).  Raises
    StoppedEarly (with the time reached) when the path reports a
    non-physical state."""
    from . import FISH_ERR_NONPHYSICAL, FishError
    steps = 0
    while t < t_end * (1.0 - 1e-12):
        try:
            dt = min(box.cfl_dt(k), 0.5 * (t_end - t))
            box.step(dt)
        except FishError as exc:
            if exc.code != FISH_ERR_NONPHYSICAL:
                raise
            raise StoppedEarly(t, steps, str(exc)) from exc
        t += 2.0 * dt
        steps += 1
        if steps > max_steps:
            raise RuntimeError("time step collapsed")
    return t, steps


def field_ranges(st, gamma, bc):
    """Ranges of density, gas pressure, magnetic energy b^2/2 and kinetic
    energy rho v^2/2 (cell-centred b: mean of the two faces)."""
    bcc = np.array(W.cell_centred(st[5:8], bc))
    e_mag = 0.5 * np.sum(bcc ** 2, axis=0)
    e_kin = 0.5 * np.sum(st[1:4] ** 2, axis=0) / st[0]
    p = (gamma - 1.0) * (st[4] - e_kin - e_mag)
    out = {}
    for key, a in (("rho", st[0]), ("p", p), ("e_mag", e_mag), ("e_kin", e_kin)):
        out[key] = (float(a.min()), float(a.max()))
    return out


def radial_profile(rho, h):
    """Mean density in shells of width h about the box centre (cubic box)."""
    n = rho.shape[-1]
    c = (np.arange(n) + 0.5) * h - 0.5 * n * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    k = np.minimum((r / h).astype(np.int64), n)
    cnt = np.bincount(k.ravel(), minlength=n + 1)
    tot = np.bincount(k.ravel(), weights=rho.ravel(), minlength=n + 1)
    prof = tot / np.maximum(cnt, 1)
    return (np.arange(n + 1) + 0.5) * h, prof


def validation(name, n=None, precision="fp32", cfl=None):
    """Run one of the paper's validation problems to its end time at the
    printed CFL number (or ``cfl``) and report value ranges."""
    from . import FISH_LIM_MINMOD, FISH_LIM_VANLEER
    gen, n0, k, lim = VALIDATION[name]
    if cfl is not None:
        k = float(cfl)
    n = int(n or n0)
    w = gen(n)
    t_end = w.meta["t_end"]
    box = Box(*w.dims, w.gamma, bc=w.bc, precision=precision, h=w.h,
              limiter=FISH_LIM_MINMOD if lim == "minmod" else FISH_LIM_VANLEER)
    box.set_state(w.state)
    out = {"report": "validation", "problem": name, "n": n, "dims": list(w.dims), "precision": precision,
           "cfl": k, "limiter": lim, "t_end": t_end}
    t0 = time.time()
    if name == "sedov":
        # the self-similar radius grows as t^(2/5): compare t_end/4 and t_end
        radii = []
        t = 0.0
        for tt in (0.25 * t_end, t_end):
            t, _ = run_to(box, tt, k, t)
            r, prof = radial_profile(box.get_state()[0], w.h[0])
            i = int(np.argmax(prof))
            radii.append(float(r[i]))
            peak = float(prof[i])
        out["shock_radius"] = {"t_end_over_4": radii[0], "t_end": radii[1], "ratio": radii[1] / radii[0],
                               "self_similar_ratio": 4.0 ** 0.4, "printed_t_end": 0.45, "cell": w.h[0]}
        out["peak_shell_density"] = peak
        out["strong_shock_density"] = (w.gamma + 1.0) / (w.gamma - 1.0)
    else:
        try:
            t, steps = run_to(box, t_end, k)
            out["double_steps"] = steps
        except StoppedEarly as exc:
            out["stopped_early"] = {"t": exc.t, "double_steps": exc.steps, "error": str(exc)[:160]}
            box.close()
            out["wall_s"] = time.time() - t0
            return out
    st = box.get_state()
    out["wall_s"] = time.time() - t0
    out["ranges"] = field_ranges(st, w.gamma, w.bc)
    if "ranges" in w.meta:
        out["printed_ranges"] = w.meta["ranges"]
    d = box.diagnostics()
    out["max_div_b"] = float(d[8])
    box.close()
    return out


def main(argv):
    what = argv[1] if len(argv) > 1 else "batch"
    t0 = time.time()
    if what == "validation":
        res = validation(argv[2], *(argv[3:4] or [None]), *(argv[4:5] or ["fp32"]),
                         *([float(argv[5])] if len(argv) > 5 else []))
        res["wall_s_total"] = time.time() - t0
        print(json.dumps(res), flush=True)
        return
    args = [int(a) for a in argv[2:]]
    res = {"polytrope": polytrope, "fp32_vs_fp64": fp32_vs_fp64, "batch": batch,
           "fp64_sweeps": fp64_sweeps, "variants": variants}[what](*args)
    res["wall_s"] = time.time() - t0
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main(sys.argv)
