"""Builds the host-C++ checks of the kernel source (tests/*.cpp) with g++ for the CPU tests."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_include():
    """Directory of cuda_runtime.h (the kernel headers include it for their host types), or None."""
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def build(src, out, shared):
    """Compile tests/<src> against the package's csrc/ and include/ into `out` (skip without g++)."""
    cxx = shutil.which("g++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    cmd = [cxx, "-std=c++17", "-O2", "-w"] + (["-shared", "-fPIC"] if shared else []) + [
        "-I" + inc, "-I" + os.path.join(ROOT, "paper_2011_02600_gb300", "csrc"),
        "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", src), "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(out)
