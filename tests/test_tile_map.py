"""CPU check of the kernels' index arithmetic: tile_map_check.cpp compiles the tiled kernel's
tile geometry (csrc/tile_map.cuh) and the row helpers of csrc/common.cuh as host C++ and checks
ownership, TMA alignment, the q rows of D- and D+ against the operator's rows, the r taps, the
launch order, apply_row, the norm weights and the SBP relation of the applied operators for
every grid size from 1 to 400 and a set of large sizes (the full-size workload's 1025 among
them)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def test_tile_geometry_for_every_grid_size(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "tile_map_check")
    build = subprocess.run([cxx, "-std=c++17", "-O2", "-w", "-I" + inc,
                            "-I" + os.path.join(ROOT, "paper_2011_02600_gb300", "csrc"),
                            "-I" + os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "tile_map_check.cpp"), "-o", exe],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stderr
