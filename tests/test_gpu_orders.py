"""The odd upwind orders 3, 5, 7 (Table 1) and the traditional central operators of orders 2,
4, 6 (Table 2) on the GPU, through the C ABI, against the FP64 oracle.

These are the operators of the paper's comparisons (Section 6.2: dispersion of even against odd
upwind orders and against the traditional operators; Section 7.2: the same on topography).  The
checks and tolerances are those of test_gpu_parity.py (1e-12 in FP64 and 5e-5 in FP32, relative
to each output field's largest magnitude); the tiled kernel is also compared with the general
one-thread-per-node kernel over ragged sizes, several s chunks and minimum sizes.
"""
import numpy as np
import pytest
import torch

from oracle import rk
from oracle.elastic import Scheme, energy, rhs
from oracle.metrics import metrics
from oracle.operators import min_nodes, traditional_min_nodes
from oracle.solver import OracleSolver
from oracle.source import PointSource, moment_tensor
from workloads.fields import gaussian_pulse, random_state, smooth_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium
from workloads.timestep import stable_dt

pytestmark = pytest.mark.gpu

MIXED = [("char", 0.0), ("char", 0.3), ("char", -0.4), ("char", 1.0), ("char", 0.0), ("free",)]
OPS = [(3, "upwind"), (5, "upwind"), (7, "upwind"), (2, "traditional"), (4, "traditional"), (6, "traditional")]
IDS = [f"{op[:4]}{o}" for o, op in OPS]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _nmin(order, operator):
    """Fewest nodes per axis: the operator's own bound and, for a traditional operator, that of
    the upwind pair of the same order, which forms the metric terms."""
    return min_nodes(order) if operator == "upwind" else max(traditional_min_nodes(order), min_nodes(order))


def _problem(nodes, order, operator, ext=(1000.0, 1100.0, 900.0)):
    X = node_coordinates(make_map("curvy", ext), nodes)
    mat = make_medium("smooth_gradient", Lz=ext[2])(*X)
    J, a = metrics(*X, order)
    return X, mat, J, a, Scheme(order, nodes, operator)


def _solver(nodes, order, operator, prec, bc, X, mat, keep=False):
    from paper_2011_02600_gb300 import ElasticSolver
    s = ElasticSolver(nodes, order, prec, bc, operator=operator)
    s.setup(torch.from_numpy(np.stack(X)), torch.from_numpy(np.stack(mat)), keep_metrics=keep)
    return s


def _relerr(got, want):
    got = np.asarray(got, dtype=float)
    axes = tuple(range(1, want.ndim))
    return (np.abs(got - want).max(axis=axes) / np.maximum(np.abs(want).max(axis=axes), 1e-300)).max()


def _idx(nodes):
    K, Jj, I = np.meshgrid(np.arange(nodes[2]), np.arange(nodes[1]), np.arange(nodes[0]), indexing="ij")
    return I, Jj, K


@pytest.mark.parametrize("order,operator", OPS, ids=IDS)
def test_metrics_and_minimum_size(order, operator):
    from paper_2011_02600_gb300 import _lib as L
    code = order + (L.SBP_TRADITIONAL if operator == "traditional" else 0)
    assert L.sbp_min_nodes(code) == _nmin(order, operator)
    nodes = (37, 19, 23)
    X, mat, J, a, _ = _problem(nodes, order, operator)
    s = _solver(nodes, order, operator, 64, MIXED, X, mat, keep=True)
    Jg, ag = s.metrics()
    assert np.abs(Jg.cpu().numpy() - J).max() / np.abs(J).max() < 1e-13
    A = np.stack([np.stack(r) for r in a])
    assert np.abs(ag.cpu().numpy() - A).max() / np.abs(A).max() < 1e-13


@pytest.mark.parametrize("order,operator", OPS, ids=IDS)
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 5e-5)])
def test_rhs_parity(order, operator, prec, tol):
    for nodes in [(41, 29, 23), (_nmin(order, operator),) * 3]:
        X, mat, J, a, sch = _problem(nodes, order, operator)
        s = _solver(nodes, order, operator, prec, MIXED, X, mat)
        if prec == 64:
            Q = random_state(nodes, 100 + order, 1.0, 1.0e6)
        else:
            Q = np.stack(smooth_state(nodes, 5, *_idx(nodes)))
        want = rhs(Q, sch, J, a, mat, MIXED)
        got = s.rhs(torch.from_numpy(Q)).cpu().numpy()
        assert _relerr(got, want) < tol, nodes


@pytest.mark.parametrize("order,operator", OPS, ids=IDS)
@pytest.mark.parametrize("nodes", [(101, 45, 40), (67, 20, 13), (65, 24, 17), (36, 12, 97), (37, 16, 200)])
@pytest.mark.parametrize("prec", [32, 64])
def test_tiled_matches_general_kernel(order, operator, nodes, prec):
    """Several tiles, ragged last tiles along q and r, closure rows split across tiles and
    several s chunks (200 planes): tiled and general kernels agree, and both match the oracle."""
    nodes = tuple(max(n, _nmin(order, operator)) for n in nodes)
    X, mat, J, a, sch = _problem(nodes, order, operator)
    s = _solver(nodes, order, operator, prec, MIXED, X, mat)
    Q = np.stack(smooth_state(nodes, 9, *_idx(nodes))) if prec == 32 else random_state(nodes, 9)
    r_tiled = s.rhs(torch.from_numpy(Q)).cpu().numpy()
    s.set_kernel_path(1)
    r_gen = s.rhs(torch.from_numpy(Q)).cpu().numpy()
    assert _relerr(r_tiled, r_gen) < (1e-12 if prec == 64 else 5e-6)
    want = rhs(Q, sch, J, a, mat, MIXED)
    assert _relerr(r_tiled, want) < (1e-12 if prec == 64 else 5e-5)


@pytest.mark.parametrize("order,operator", OPS, ids=IDS)
@pytest.mark.parametrize("stage", [0, 3])
def test_fused_stage_and_energy_fp64(order, operator, stage):
    nodes = (37, 19, 14) if _nmin(order, operator) <= 14 else (37, 19, 16)
    X, mat, J, a, sch = _problem(nodes, order, operator)
    s = _solver(nodes, order, operator, 64, MIXED, X, mat)
    Q = random_state(nodes, 31, 1.0, 1.0e6)
    dQ = random_state(nodes, 32, 0.1, 1.0e5)
    s.set_state(torch.from_numpy(Q), reset_register=False)
    assert abs(s.energy() - energy(Q, sch, J, mat)) <= 1e-12 * energy(Q, sch, J, mat)
    s.view(s.dq, 9).copy_(torch.from_numpy(dQ))
    dt = 2.5e-3
    s.rk_stage(stage, dt)
    L = rhs(Q, sch, J, a, mat, MIXED)
    dq_new = (rk.A[stage] * dQ if stage else 0.0) + dt * L
    q_new = Q + rk.B[stage] * dq_new
    assert _relerr(s.view(s.dq, 9).cpu().numpy(), dq_new) < 1e-12
    assert _relerr(s.state().cpu().numpy(), q_new) < 1e-12


@pytest.mark.parametrize("order,operator", OPS, ids=IDS)
def test_all_free_surface_energy_rate_gpu(order, operator):
    """Section 5.1: with the free-surface penalty on every face, <Q, P~^-1 dQ/dt>_H = 0 for the
    GPU's own right-hand side (both the upwind pairs and the traditional operators are SBP)."""
    nodes = (41, 29, 23)
    X, mat, J, a, sch = _problem(nodes, order, operator)
    s = _solver(nodes, order, operator, 64, [("free",)] * 6, X, mat)
    Q = random_state(nodes, 7, 1.0, 1.0)
    d = s.rhs(torch.from_numpy(Q)).cpu().numpy()
    rho, lam, mu = mat
    W = sch.weights3()
    pv = sum(Q[c] * rho * J * d[c] for c in range(3))
    ds = d[3:9]
    tr = ds[0] + ds[1] + ds[2]
    Sd = [(ds[c] - lam / (3 * lam + 2 * mu) * tr) / (2 * mu) for c in range(3)] + [ds[c] / mu for c in range(3, 6)]
    ps = sum(Q[3 + c] * J * Sd[c] for c in range(6))
    val = float(np.sum(W * (pv + ps)))
    scale = float(np.sum(np.abs(W * pv)))
    assert abs(val) < 1e-12 * scale


@pytest.mark.parametrize("order,operator", [(5, "upwind"), (6, "traditional")], ids=["upwi5", "trad6"])
def test_source_run_against_oracle(order, operator):
    """Moment-tensor source (Ricker) on a curvilinear grid, FP64, 30 steps, 3 receivers; the
    source's moment conditions follow the operator's design order."""
    import math
    nodes = (29, 27, 25)
    X, mat, J, a, sch = _problem(nodes, order, operator, ext=(2000.0, 2000.0, 1500.0))
    bc = [("char", 0.0)] * 5 + [("free",)]
    dt = stable_dt(*X, *mat, 0.5)
    Mv = moment_tensor(0.3, 1.1, -0.7, 1.0e13)
    ref = (0.43, 0.52, 0.61)
    f0 = 25.0

    def ricker(t):
        x = (math.pi * f0 * (t - 1.2 / f0)) ** 2
        return (1 - 2 * x) * math.exp(-x)
    orc = OracleSolver(order, *X, mat, bc, operator=operator)
    orc.sources.append(PointSource(ref, Mv, ricker, order, nodes, sch.weights3(), J))
    rec = [(10, 12, 24), (20, 5, 24), (14, 14, 12)]
    orc.receivers = rec
    orc.step(dt, 30)
    s = _solver(nodes, order, operator, 64, bc, X, mat, keep=True)
    s.set_source(ref, Mv, "ricker", f0=f0)
    tr = s.set_receivers(rec, 30)
    s.step(30, dt)
    assert _relerr(s.state().cpu().numpy(), orc.Q) < 1e-11
    want = np.stack(orc.traces, axis=-1)
    assert np.abs(tr.cpu().numpy() - want).max() / np.abs(want).max() < 1e-11


@pytest.mark.parametrize("order,operator", [(7, "upwind"), (4, "traditional")], ids=["upwi7", "trad4"])
def test_pulse_run_fp32_against_fp64_oracle(order, operator):
    """FP32 run of a pulse on a curvilinear grid over 40 steps against the FP64 oracle, relative
    to the peak amplitude (the FP32 target of 1e-4)."""
    nodes = (41, 29, 23)
    X, mat, J, a, sch = _problem(nodes, order, operator, ext=(4000.0, 2800.0, 2200.0))
    bc = [("char", 0.0)] * 5 + [("free",)]
    dt = stable_dt(*X, *mat, 0.5)
    Q0 = np.stack(gaussian_pulse(*X, (2000.0, 1400.0, 1100.0), 250.0))
    orc = OracleSolver(order, *X, mat, bc, operator=operator)
    orc.Q[:] = Q0
    orc.step(dt, 40)
    s = _solver(nodes, order, operator, 32, bc, X, mat)
    s.set_state(torch.from_numpy(Q0))
    s.step(40, dt)
    got = s.state().cpu().numpy().astype(float)
    err = np.abs(got[:3] - orc.Q[:3]).max() / np.abs(orc.Q[:3]).max()
    assert err < 1e-4, err


@pytest.mark.parametrize("order,operator", [(3, "upwind"), (2, "traditional")], ids=["upwi3", "trad2"])
def test_adjoint_refused(order, operator):
    """The adjoint kernels are built for the even upwind orders only: the C ABI says so."""
    from paper_2011_02600_gb300 import _lib as L
    nodes = (20, 20, 20)
    X, mat, J, a, sch = _problem(nodes, order, operator)
    s = _solver(nodes, order, operator, 64, MIXED, X, mat)
    w, out, scr = s.new_fields(9), s.new_fields(9), s.new_fields(9)
    with pytest.raises(L.SbpError) as e:
        L.sbp_rhs_adjoint(s.h, w, out, scr, 0)
    assert e.value.code == 2
