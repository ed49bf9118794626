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


@pytest.mark.parametrize("order,nodes", [(4, (45, 33, 30)), (6, (40, 27, 31)), (2, (35, 20, 18))])
@pytest.mark.parametrize("precision", [64, 32])
def test_adjoint_passes_on_topography_path(order, nodes, precision):
    """The adjoint's tiled passes on the topography path against the general path: L^T w
    (sbp_rhs_adjoint) and one adjoint stage with its material gradient (sbp_adjoint_stage)."""
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    from paper_2011_02600_gb300.workload_setup import build_solver
    from workloads.fields import random_state
    cfg = dataclasses.replace(config_by_name("adjoint129_o4"), nodes=nodes, order=order)
    s, info = build_solver(cfg, precision=precision, keep_metrics=True)
    assert s.map_path() == "topography"
    st = _stream()
    rlmj = s.new_fields(4, torch.float64)
    r = s.view(rlmj, 4)
    J = s.view(s.jmet, 10)[0]
    mat = s.view(s.mat, 3).double()
    r[3].copy_(J)
    r[0].copy_(1.0 / (mat[0] * J))
    r[1].copy_(mat[1] * J)
    r[2].copy_(mat[2] * J)
    y = s.to_layout(torch.from_numpy(random_state(nodes, 71, 1.0e-6, 1.0)), s.dtype)
    u = s.to_layout(torch.from_numpy(random_state(nodes, 72, 1.0, 1.0e6)), s.dtype)
    ub0 = s.to_layout(torch.from_numpy(random_state(nodes, 73, 1.0e-6, 1.0)), s.dtype)
    wb0 = s.to_layout(torch.from_numpy(random_state(nodes, 74, 1.0e-6, 1.0)), s.dtype)
    out = {}
    for path in ("auto", "general"):
        s.set_map_path(path)
        lt, scratch = s.new_fields(9), s.new_fields(9)
        L.sbp_rhs_adjoint(s.h, y, lt, scratch, st)
        ub, wb, grad = ub0.clone(), wb0.clone(), s.new_fields(3, torch.float64)
        L.sbp_adjoint_stage(s.h, 2, info["dt"], u, ub, wb, scratch, rlmj, grad, st)
        torch.cuda.synchronize()
        out[path] = [s.view(x, n).double().cpu().numpy() for x, n in ((lt, 9), (ub, 9), (wb, 9), (grad, 3))]
    tol = 1e-12 if precision == 64 else 1e-5
    for a, b in zip(out["auto"], out["general"]):
        scale = np.abs(b).max(axis=(1, 2, 3))
        assert scale.min() > 0
        assert (np.abs(a - b).max(axis=(1, 2, 3)) / scale).max() < tol
