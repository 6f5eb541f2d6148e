"""CPU checks of the C ABI: the library builds, loads and exports every
symbol include/fish.h declares; the binding fails loudly without it."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "fish.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fish_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0910_2854_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fish_\w+)", out))
    declared = declared_symbols()
    assert declared, "no declarations parsed"
    assert set(declared) <= exported, set(declared) - exported


def test_binding_lists_every_declared_symbol(libpath):
    import paper_0910_2854_gb300 as F
    assert sorted(F.EXPORTS) == declared_symbols()
    lib = F.load(libpath)
    for name in F.EXPORTS:
        assert hasattr(lib, name)


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_0910_2854_gb300 as F
    saved = F._lib
    F._lib = None
    try:
        with pytest.raises(F.FishError):
            F.load(str(tmp_path / "missing.so"))
    finally:
        F._lib = saved


def test_kernels_compile_for_sm103a_with_small_spills_in_fp32(libpath):
    """The FP32 sweep kernels are register-capped for occupancy; what spills
    to local memory (served by L1) must stay small."""
    from paper_0910_2854_gb300 import build
    cmd = [build.nvcc(), "-c", os.path.join(build.CSRC, "fish_f32.cu"), "-o", os.devnull] + build.ARCH + \
        build.COMMON + ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True, check=True)
    out = r.stdout + r.stderr
    blocks = re.findall(r"Function properties for (\w+)\n\s+(\d+) bytes stack frame, (\d+) bytes spill stores", out)
    assert blocks
    for name, stack, spill in blocks:
        if "sweep" in name:
            assert int(spill) <= 512, (name, spill)
