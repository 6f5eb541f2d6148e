#!/usr/bin/env python
"""Throughput of FISH's operator-split ideal-MHD double step on GB300.

Metric: MHD cell-updates/s per full x-y-z-z-y-x double step (cells / step
time, the step including the device CFL reduction), FP32 path on the
1024^3 random-phase turbulence box, with the FP64 path on the 256^3
Orszag-Tang box reported beside it, and the HBM roofline fraction of the
dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fish|reference]

N > 1 runs as one rank per GPU under torch.distributed.run; every rank
advances its own box (independent replicas, no collective on the data
path), so scaling is weak and the value is the cells of all ranks divided by
the slowest rank's time.  With --decomp the ranks instead share one box split
into z-slabs (ghost planes exchanged before every operator, all-reduced CFL
step; strong scaling, the value is the box's cells over the slowest rank's
time).  ``--impl reference`` times the CPU oracle (the
FP64 C implementation in oracle/) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MHD cell-updates/s per full xyzzyx step"
UNIT = "cell-updates/s"
CFL = 0.5
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

WORKLOAD = {
    "workload": "random-phase MHD turbulence 1024^3 periodic, FP32 bulk with compensated pressure "
                "recovery and FP64 reductions (k^-2 spectrum, |k|<=8, rms Mach 1, beta 1, rho=1, p=1, "
                "seeds 910285/910286)",
    "n": 1024,
    "precision": "fp32",
    "gamma": 5.0 / 3.0,
}


def workload_name(n):
    """The workload's description at n^3 cells (1024^3 is the timed box)."""
    return WORKLOAD["workload"].replace("1024^3", "%d^3" % n)


def l2_note(n):
    """Whether one copy of the FP32 state (32 B per cell) exceeds the 129 MB L2."""
    gb = 32.0 * n ** 3 / 1e9
    if gb * 1e3 > 129.0:
        return "inputs larger than L2 (%.3g GB state vs 129 MB L2)" % gb
    return "inputs fit in L2 (%.3g MB state vs 129 MB L2): small test size, not a timing configuration" % (gb * 1e3)


FP64_WORKLOAD = {
    "workload": "3D Orszag-Tang-type vortex 256^3 periodic, FP64 (plain method)",
    "n": 256,
    "precision": "fp64",
}
# algorithmic bytes per cell of one launch (state fields the operator must
# read and write, one word each): L_d reads 8 fields and writes 5, B_d reads
# rho, m_d and 3 field components and writes 3.
ALG_WORDS = {"fluid": 13, "ct": 8}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="fish", choices=("fish", "reference"))
    p.add_argument("--n", type=int, default=None, help="override the box size (testing)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--kernels", default="column", choices=("column", "ring"),
                   help="kernel family of the FP32 fluid sweep: register-prefetch column march (default) or the "
                        "march fed through a shared-memory ring of TMA bulk copies")
    p.add_argument("--decomp", action="store_true",
                   help="one box split into z-slabs over the ranks (halo exchange, strong scaling) instead of one "
                        "box per rank")
    p.add_argument("--no-same-box", action="store_true",
                   help="skip the FP64 run of the workload's own box (like-for-like FP32/FP64 ratio and L1(rho))")
    p.add_argument("--oracle-sample", type=float, default=None,
                   help="print only the oracle's rate on the 128^3 twin within this many seconds (the "
                        "single-core leg runs itself this way with OMP_NUM_THREADS=1)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.count(",") >= 8]
        try:
            os.unlink(self.tmp.name)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = [nm for i, nm in enumerate(names) if any(r[5 + i].strip() == "Active" for r in rows)]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
# The coarse twins of the turbulence box resolve its shortest waves (k = 8)
# with 16 cells at 128^3: there the method reaches p < 0 after about ten
# double steps (the 1024^3 box stays physical), so timed oracle samples
# restart from the initial state every RESTART_STEPS steps.
RESTART_STEPS = 6


def oracle_rate(n_twin=128, budget_s=10.0, min_steps=1, max_steps=50):
    """Oracle cell-updates/s on the 128^3 twin of the turbulence box: whole
    double steps (CFL included) until ``budget_s`` of CPU time, the state
    restarted (outside the timed region) every RESTART_STEPS steps."""
    import oracle
    from paper_0910_2854_gb300 import workloads as W
    oracle.build()
    w = W.turbulence(n_twin)
    ob = oracle.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h)
    ob.set_state(w.state)
    el = 0.0
    steps = 0
    while steps < min_steps or (el < budget_s and steps < max_steps):
        if steps and steps % RESTART_STEPS == 0:
            ob.set_state(w.state)
        t0 = time.perf_counter()
        ob.step(ob.cfl(CFL))
        el += time.perf_counter() - t0
        steps += 1
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return w.ncells * steps / el, steps, el, cores, w.ncells


def oracle_rate_single_core(budget_s=8.0):
    """The same oracle sample on one host core (a child process with
    OMP_NUM_THREADS=1, so the OpenMP runtime of this process is untouched)."""
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(budget_s)],
                         env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    sample = 128 if args.n is None else min(args.n, 128)
    # warm-up steps (untimed), then K timed steps on the bounded sample
    rate_w, _, _, _, _ = oracle_rate(sample, budget_s=0.0, min_steps=max(1, min(args.warmup, 2)), max_steps=2)
    import oracle
    from paper_0910_2854_gb300 import workloads as W
    w = W.turbulence(sample)
    ob = oracle.OracleBox(*w.dims, w.gamma, bc=w.bc, h=w.h)
    ob.set_state(w.state)
    el = 0.0
    for k in range(args.steps):
        if k and k % RESTART_STEPS == 0:
            ob.set_state(w.state)  # outside the timed region, see RESTART_STEPS
        t0 = time.perf_counter()
        ob.step(ob.cfl(CFL))
        el += time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = w.ncells * args.steps / el
    cfg = {"workload": WORKLOAD["workload"], "sample": "%d^3 twin of the workload" % sample,
           "precision": "fp64 (oracle)", "cfl": CFL}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d double steps of the %d^3 twin, restarted every %d steps"
                                       % (args.steps, sample, RESTART_STEPS)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def make_box(F, W, spec, n, torch, kernels="column"):
    prec = spec["precision"]
    dt_ = torch.float32 if prec == "fp32" else torch.float64
    if spec is WORKLOAD:
        w = W.turbulence(n, device="cuda", dtype=dt_)
        st = w.state
    else:
        w = W.orszag_tang(n)
        st = torch.as_tensor(w.state, device="cuda", dtype=dt_)
    box = F.Box(n, n, n, w.gamma, precision=prec, h=w.h, kernels=kernels)
    box.set_state(st)
    del st, w
    torch.cuda.empty_cache()
    return box


def time_steps(box, torch, steps, warmup):
    box.step_cfl(CFL, warmup)
    box.sync()
    s = box.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = box.launch_count()
    e0.record(s)
    box.step_cfl(CFL, steps)
    e1.record(s)
    e1.synchronize()
    box.sync()
    return e0.elapsed_time(e1), box.launch_count() - l0


def time_operators(F, box, torch, reps=3):
    """Average duration of each operator kind (CUDA events on the library's
    stream), with the dt of the current state.  Every kind starts from the
    same state (a device snapshot): repeating one directional operator is
    not the method's composition and would drift the state."""
    dt = box.cfl_dt(CFL)
    s = box.stream
    n = box.n[0] * box.n[1] * box.n[2]
    snap = torch.empty(8 * n, dtype=torch.float32 if box.precision == "fp32" else torch.float64, device="cuda")
    box.get_state_device(snap)
    out = {}
    for kind, op in (("fluid", F.FISH_OP_FLUID), ("ct", F.FISH_OP_CT)):
        for d in range(3):
            # the repeated operator may leave a non-physical state behind on
            # coarse boxes; the restored snapshot replaces it
            box.sync_quiet()
            box.set_state(snap)
            box.apply(op, d, dt)  # warm
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                box.apply(op, d, dt)
            e1.record(s)
            e1.synchronize()
            out["%s_%s" % (kind, "xyz"[d])] = e0.elapsed_time(e1) / reps
    box.sync_quiet()
    box.set_state(snap)
    del snap
    torch.cuda.empty_cache()
    return out


# DRAM bytes per cell of one launch of each kernel kind, from the ncu
# capture of the 384^3 turbulence box (dram__bytes_read.sum +
# dram__bytes_write.sum over its cells).  Set an entry to None when that
# kernel changes until it is captured again.
TRAFFIC_B_PER_CELL = {"fluid": 52.1, "ct": 32.1}


# FP64 pipe instructions (DADD + DMUL + DFMA, thread level) per cell of one
# launch of each FP64 kernel kind, from the ncu capture of the Orszag-Tang
# 128^3 box.  The FP64 path
# is bound by GB300's FP64 pipe, so its roofline is this rate against the
# probed FMA rate of the device (fish_probe_fp64_fma).
FP64_OPS_PER_CELL = {"fluid": 537, "ct": 170}


def traffic_per_cell(kernel_key):
    return TRAFFIC_B_PER_CELL.get(kernel_key.split("_")[0])


def e2e_rate(F, box, torch, n, steps):
    """End to end through the public API, a full host round trip per step:
    upload the whole state from pinned host memory (fish_set_state_host,
    FP32, the path's arithmetic type), advance one double step with the
    device CFL, and download the whole new state into the same pinned buffer
    (fish_get_state_host, which also returns any device error)."""
    N = n ** 3
    host = torch.empty((8, n, n, n), dtype=torch.float32, pin_memory=True)
    box.get_state_host(host)
    t0 = time.perf_counter()
    for _ in range(steps):
        box.set_state_host(host)
        box.step_cfl(CFL, 1)
        box.get_state_host(host)
    el = time.perf_counter() - t0
    del host
    return N * steps / el, 32 * N, 32 * N


def run_fish(args, rank, world, local):
    import torch
    import paper_0910_2854_gb300 as F
    from paper_0910_2854_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.n or WORKLOAD["n"]
    box = make_box(F, W, WORKLOAD, n, torch, args.kernels)
    clocks = ClockSampler(local)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    clocks.start()
    ms, launches = time_steps(box, torch, args.steps, args.warmup)
    barrier()
    clk = clocks.stop()
    # cells of all ranks over the slowest rank's time (every rank its own box)
    from paper_0910_2854_gb300.replicas import job_throughput
    rate, ms = job_throughput(ms, n ** 3 * args.steps, device="cuda")
    ms_step = ms / args.steps
    value = rate

    result = None
    if rank == 0:
        ops = time_operators(F, box, torch)
        key = max(ops, key=ops.get)
        kind = key.split("_")[0]
        esz = 4 if WORKLOAD["precision"] == "fp32" else 8
        alg = ALG_WORDS[kind] * esz * n ** 3
        peak, peak_kind = measured_peak()
        achieved = alg / (ops[key] * 1e-3) / 1e9
        tpc = traffic_per_cell(key)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if tpc is None else tpc * n ** 3, "kernel": key,
                "kernel_ms": ops[key], "peak_source": peak_kind,
                "step_alg_GBs": 384 * n ** 3 / (ms_step * 1e-3) / 1e9,
                "step_frac": 384 * n ** 3 / (ms_step * 1e-3) / 1e9 / peak,
                "op_ms": ops}
        e2e = None
        if not args.no_e2e:
            try:
                ev, hb, db = e2e_rate(F, box, torch, n, max(2, min(args.steps, 5)))
                e2e = {"value": ev, "unit": UNIT, "h2d_bytes_per_step": hb, "d2h_bytes_per_step": db}
            except Exception as exc:  # report, do not hide
                e2e = {"value": None, "unit": UNIT, "error": repr(exc)[:200]}
        box.close()
        torch.cuda.empty_cache()
        fp64 = None
        if not args.no_fp64:
            b64 = make_box(F, W, FP64_WORKLOAD, FP64_WORKLOAD["n"], torch)
            ms64, _ = time_steps(b64, torch, max(3, min(args.steps, 10)), args.warmup)
            k64 = max(3, min(args.steps, 10))
            n64 = FP64_WORKLOAD["n"] ** 3
            v64 = n64 / (ms64 / k64 * 1e-3)
            ops64 = time_operators(F, b64, torch)
            key64 = max(ops64, key=ops64.get)
            peak64 = F.probe_fp64_fma()
            ach64 = FP64_OPS_PER_CELL[key64.split("_")[0]] * n64 / (ops64[key64] * 1e-3)
            fp64 = {"workload": FP64_WORKLOAD["workload"], "value": v64, "unit": UNIT, "ms_per_step": ms64 / k64,
                    "fp32_turbulence_over_fp64_orszag_tang": (value / world) / v64,
                    "roofline": {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "FP64 pipe op/s",
                                 "frac": ach64 / peak64, "kernel": key64, "kernel_ms": ops64[key64],
                                 "ops_per_cell": FP64_OPS_PER_CELL[key64.split("_")[0]],
                                 "peak_source": "probed (fish_probe_fp64_fma)", "op_ms": ops64}}
            b64.close()
            torch.cuda.empty_cache()
            if not args.no_same_box:
                # like for like: the same turbulence box advanced in FP64 (3
                # double steps each way from the same initial state)
                from paper_0910_2854_gb300 import reports
                sb = reports.fp32_vs_fp64(n, steps=3, k=CFL)
                fp64["same_box"] = {
                    "workload": workload_name(n).replace("FP32 bulk with compensated pressure recovery and "
                                                         "FP64 reductions", "FP64 throughout"),
                    "fp64_ms_per_step": sb["fp64"]["ms_per_step"], "fp64_value": sb["fp64"]["cell_updates_per_s"],
                    "fp32_over_fp64": (value / world) / sb["fp64"]["cell_updates_per_s"],
                    "l1_rho_rel_fp32_vs_fp64": sb["l1_rho_rel"], "steps_compared": 3}
                torch.cuda.empty_cache()
        batch = None
        if not args.no_batch:
            from paper_0910_2854_gb300 import reports
            try:
                batch = reports.batch()
                peak_b, _ = measured_peak()
                # the method's floor (384 B/cell per double step) at the batch's rate
                batch["step_frac"] = 384 * batch["cells"] / (batch["ms_per_step"] * 1e-3) / 1e9 / peak_b
                batch["workload"] = ("batch of 64 seeded boxes 32^3..160^3 (Sod / Brio-Wu / blast), FP32, one graph "
                                     "of persistent work-queue sweeps per double step, autotuned")
            except Exception as exc:  # report, do not hide
                batch = {"error": repr(exc)[:200]}
        cpu = None
        if not args.no_cpu_baseline:
            rate, steps, el, cores, cells = oracle_rate(128, budget_s=10.0)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d double steps (%.1f s) of the 128^3 twin (%d cells) of the workload, "
                             "restarted every %d steps" % (steps, el, cells, RESTART_STEPS)}
            try:
                cpu["single_core"] = oracle_rate_single_core(8.0)
            except Exception as exc:  # report, do not hide
                cpu["single_core"] = {"error": repr(exc)[:200]}
        result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                  "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                  "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded, generated on the device)",
                  "config": {"workload": workload_name(n), "cells": n ** 3, "cfl": CFL,
                             "parallelism": "replicas x%d (one box per GPU, no data-path collective)" % world,
                             "l2": l2_note(n),
                             "graph": "one CUDA graph per double step (CFL + 12 sweeps)",
                             "fluid_kernels": args.kernels},
                  "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                  "clocks": clk, "fp64_path": fp64, "batch": batch}
    else:
        box.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


def run_fish_decomp(args, rank, world, local):
    """One n^3 turbulence box split into z-slabs over the ranks (host-driven
    operators with a ghost-plane exchange before each, no graph)."""
    import torch
    import paper_0910_2854_gb300 as F
    from paper_0910_2854_gb300 import decomp
    from paper_0910_2854_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.n or WORKLOAD["n"]
    k0, nk, lo, hi = decomp.slab_extent(n, rank, world, True)
    w = W.turbulence(n, device="cuda", dtype=torch.float32)
    idx = torch.arange(k0 - lo, k0 + nk + hi, device="cuda") % n
    slab = w.state.view(8, n, n, n).index_select(1, idx).contiguous()
    gamma, h = w.gamma, w.h
    del w
    torch.cuda.empty_cache()
    box = F.Box(n, n, lo + nk + hi, gamma, precision="fp32", h=h)
    box.set_state(slab)
    del slab
    torch.cuda.empty_cache()
    run = decomp.SlabRun(box, n, n, n, rank, world, periodic=True, dist=dist, device="cuda", dtype=torch.float32)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    run.step_cfl(CFL, args.warmup)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = box.launch_count()
    e0.record(box.stream)
    run.step_cfl(CFL, args.steps)
    e1.record(box.stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = box.launch_count() - l0
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = n ** 3 / (ms_step * 1e-3)
    box.close()
    if rank == 0:
        peak, peak_kind = measured_peak()
        per_gpu = 384 * n ** 3 / world / (ms_step * 1e-3) / 1e9
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded, generated on the device)",
                "config": {"workload": workload_name(n), "cells": n ** 3, "cfl": CFL,
                           "parallelism": "z-slabs x%d (%d ghost planes exchanged before every operator, "
                                          "all-reduced CFL step)" % (world, decomp.HALO),
                           "l2": l2_note(n)},
                "roofline": {"bound": "hbm", "achieved": per_gpu, "peak": peak, "unit": "GB/s",
                             "frac": per_gpu / peak, "traffic": None,
                             "kernel": "whole double step per GPU (384 B/cell floor)", "peak_source": peak_kind},
                "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
                "exchanges_per_step": run.exchanges / (args.steps + args.warmup)}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.oracle_sample is not None:
        rate, steps, el, cores, cells = oracle_rate(128, budget_s=args.oracle_sample)
        print(json.dumps({"value": rate, "unit": UNIT, "cores": cores, "steps": steps, "seconds": el}))
        return 0
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.decomp:
        return run_fish_decomp(args, rank, world, local)
    return run_fish(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
