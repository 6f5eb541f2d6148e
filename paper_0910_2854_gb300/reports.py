"""Measurements of the GPU path beyond the throughput line of bench.py, run
on one GPU and printed as one JSON line each:

  python -m paper_0910_2854_gb300.reports polytrope [n] [steps]
      n = 1 polytrope (n^3, FP32 with the hydrostatic island) with and
      without the hydrostatic-gradient correction: central density drift
      and largest spurious velocity after `steps` double steps.
  python -m paper_0910_2854_gb300.reports fp32_vs_fp64 [n] [steps]
      random-phase turbulence n^3: FP32 and FP64 paths each advanced with
      their own CFL steps; L1 density difference relative to the FP64 path,
      and both throughputs.
  python -m paper_0910_2854_gb300.reports batch
      the seeded batch of 64 uneven boxes: autotuned choice and throughput.

Every step runs in the CUDA kernels behind the C ABI; the inputs are the
seeded synthetic fields of ``workloads``.
"""
from __future__ import annotations

import json
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


def polytrope(n=384, steps=1000, k=0.5):
    import torch
    w = W.polytrope(n)
    c = n // 2
    out = {"report": "polytrope", "n": n, "steps": steps, "cfl": k, "precision": "fp32",
           "rho_c0": float(w.state[0, c, c, c])}
    for hse in (False, True):
        box = Box(*w.dims, w.gamma, bc=w.bc, precision="fp32", h=w.h, hse=hse)
        box.set_state(w.state)
        box.set_potential(w.phi)
        t = 0.0
        ms = 0.0
        for _ in range(steps // 50):
            ms += _timed_steps(box, torch, k, 50)
            t += 2 * 50 * box.last_dt()  # approximate: the last dt of each chunk
        st = box.get_state()
        v = np.sqrt(st[1] ** 2 + st[2] ** 2 + st[3] ** 2) / st[0]
        inside = w.state[0] > 10 * w.state[0].min()
        key = "hse" if hse else "no_hse"
        out[key] = {"rho_c": float(st[0, c, c, c]),
                    "rho_c_drift": float(st[0, c, c, c] / out["rho_c0"] - 1.0),
                    "vmax_star": float(v[inside].max()), "vmax": float(v.max()),
                    "ms_per_step": ms / steps, "t_approx": t}
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
           "tuning": {kk: choice[kk] for kk in ("order", "groups", "grid")}}
    b.close()
    return out


def main(argv):
    what = argv[1] if len(argv) > 1 else "batch"
    args = [int(a) for a in argv[2:]]
    t0 = time.time()
    res = {"polytrope": polytrope, "fp32_vs_fp64": fp32_vs_fp64, "batch": batch}[what](*args)
    res["wall_s"] = time.time() - t0
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main(sys.argv)
