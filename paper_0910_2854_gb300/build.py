"""Build libfish.so in-tree with nvcc for sm_103a (GB300).

Three translation units compiled in parallel, then linked:
  fish_f64.cu  -- FP64 kernels, -fmad=false (IEEE rounding of each operation)
  fish_f64_t2.cu -- the FP64 sweeps with the fast axis t2, same flags
  fish_f32.cu  -- FP32 kernels (FMA contraction allowed)
  fish_p2.cu   -- FP32 two-column sweep kernels (packed FP32x2), Van Leer
  fish_p2_mm.cu, fish_p2_hy.cu -- the same with the minmod / hybrid limiter
  fish_capi.cu -- host-side C ABI
  fish_noalloc.cu -- the allocation-free diagnostics entry point
  fish_batch.cu -- batches of independent boxes (FP32)
  fish_ring.cu -- FP32 sweeps fed through a shared-memory ring of bulk copies
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfish.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(os.path.dirname(HERE), "include")]
UNITS = {
    "fish_f64.cu": ["-fmad=false"],
    "fish_f64_t2.cu": ["-fmad=false"],
    "fish_f32.cu": ["-prec-sqrt=false", "-ftz=true"],
    "fish_p2.cu": ["-prec-sqrt=false", "-ftz=true"],
    "fish_p2_mm.cu": ["-prec-sqrt=false", "-ftz=true"],
    "fish_p2_hy.cu": ["-prec-sqrt=false", "-ftz=true"],
    "fish_capi.cu": [],
    "fish_noalloc.cu": [],
    "fish_batch.cu": ["-prec-sqrt=false", "-ftz=true"],
    "fish_ring.cu": ["-prec-sqrt=false", "-ftz=true"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    out.append(os.path.join(os.path.dirname(HERE), "include", "fish.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False, extra=(), lib=None) -> str:
    """Compile the library (to ``lib``, default _build/libfish.so); ``extra``
    nvcc flags are added to every unit (e.g. -D tuning macros)."""
    out_lib = lib or LIB
    if not force and lib is None and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    tag = "" if lib is None else "_" + os.path.basename(out_lib).replace(".so", "")
    for unit, flags in UNITS.items():
        obj = os.path.join(BUILD, unit.replace(".cu", tag + ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, unit), "-o", obj] + ARCH + COMMON + flags + list(extra)
        if verbose:
            print(" ".join(cmd))
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(unit)
    if failed:
        raise RuntimeError("nvcc failed for %s" % ", ".join(failed))
    tmp = out_lib + ".%d.tmp" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_lib)
    return out_lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
