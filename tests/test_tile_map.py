"""CPU check of the kernels' index arithmetic: tile_map_check.cpp compiles the tiled kernel's
tile geometry (csrc/tile_map.cuh) and the row helpers of csrc/common.cuh as host C++ and checks
ownership, TMA alignment, the q rows of D- and D+ against the operator's rows, the r taps, the
launch order, the closure-row sums along s, apply_row, the norm weights and the SBP relation of
the applied operators for
every grid size from 1 to 400 and a set of large sizes (the full-size workload's 1025 among
them)."""
import subprocess

from host_build import build


def test_tile_geometry_for_every_grid_size(tmp_path):
    exe = build("tile_map_check.cpp", tmp_path / "tile_map_check", shared=False)
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stderr
