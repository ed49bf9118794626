"""The tiled forward stage's topography-map path (sbp_set_map_path, sbp_map_path): on the
layered Gaussian-hill and sinusoidal-topography grids (x = L_x q, y = L_y r, z = z(q, r, s))
a_q and a_r have one component each, and the stage reads a_q,x and a_s only.  It must give the
general path's results: the metric components it leaves out are zero up to the rounding of
D_c applied to the linear x and y, and the remaining products are the same.

* the path is chosen on those grids for the upwind orders 2, 4, 6, and not on a curvilinear map
  nor for the orders without the variant;
* state after steps with a moment source on the topography and the general path: FP64 to 1e-12
  and FP32 to 1e-5 of the fields' peaks (FP32 rounding of a different product order);
* the full-grid FP64 hill workload against the oracle (test_gpu_workloads) runs on this path.
"""
import dataclasses

import numpy as np
import pytest
import torch

from workloads.configs import config_by_name

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _run(cfg, precision, path, steps):
    from paper_2011_02600_gb300.source_util import moment_tensor_voigt
    from paper_2011_02600_gb300.workload_setup import build_solver
    s, info = build_solver(cfg, precision=precision, keep_metrics=True)
    s.set_map_path(path)
    chosen = s.map_path()
    Mv = moment_tensor_voigt(30.0, 60.0, 90.0, 1.0e15)
    s.set_source((0.5, 0.5, 0.6), Mv, "ricker", f0=cfg.extra.get("f0", 2.0))
    s.step(steps, info["dt"])
    assert s.status() == 0
    return s.state().double().cpu().numpy(), chosen


CASES = [("hill129_o6", (65, 57, 49), 6), ("hill129_o6", (61, 45, 40), 4), ("topo1025_o6_fp32", (97, 81, 41), 6),
         ("topo1025_o6_fp32", (45, 50, 33), 2)]


@pytest.mark.parametrize("name,nodes,order", CASES)
@pytest.mark.parametrize("precision", [64, 32])
def test_topography_path_matches_general(name, nodes, order, precision):
    cfg = dataclasses.replace(config_by_name(name), nodes=nodes, order=order)
    if cfg.extra.get("f0") is None:
        cfg = dataclasses.replace(cfg, extra=dict(cfg.extra, f0=2.0))
    steps = 30
    a, pa = _run(cfg, precision, "auto", steps)
    b, pb = _run(cfg, precision, "general", steps)
    assert pa == "topography" and pb == "general"
    peak = np.abs(b).max(axis=(1, 2, 3))
    assert peak.min() > 0
    err = (np.abs(a - b).max(axis=(1, 2, 3)) / peak).max()
    tol = 1e-12 if precision == 64 else 1e-5
    print(f"{name} {nodes} order {order} FP{precision}: topography vs general {err:.2e}")
    assert err < tol, err


def test_path_not_chosen_off_topography_maps():
    from paper_2011_02600_gb300 import ElasticSolver
    from workloads.geometry import make_map, node_coordinates
    from workloads.media import make_medium
    nodes = (41, 37, 33)
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    s = ElasticSolver(nodes, 6, 32, [("free",)] * 6)
    s.setup(np.stack(X), np.stack(mat))
    assert s.map_path() == "general"
    # a topography map with an order that has no topography variant, and the general kernel path
    cfg = dataclasses.replace(config_by_name("hill129_o6"), nodes=(41, 37, 33), order=5)
    from paper_2011_02600_gb300.workload_setup import build_solver
    t, _ = build_solver(cfg, precision=32)
    assert t.map_path() == "general"
    u, _ = build_solver(dataclasses.replace(cfg, order=4), precision=32)
    assert u.map_path() == "topography"
    u.set_kernel_path(1)
    assert u.map_path() == "general"
    u.set_kernel_path(0)
    u.set_map_path("general")
    assert u.map_path() == "general"
