"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
* FP64 kernels: 1e-12 relative to the largest magnitude of each output field
  (the stated target for GPU FP64 against the oracle).
* FP32 kernels: 5e-5 relative to the largest magnitude of each output field.
  Derivation: every input is rounded to FP32 (relative 6e-8); a D+- row sums at
  most 10 terms with coefficients of magnitude <= 5, scaled by N-1 <= 1024, so
  rounding noise in the inputs reaches the derivatives with a factor of at most
  ~5e3 relative to the smooth signal's derivative amplitude on the sizes used
  here (>= 2e-5 would be hit only by adversarial inputs); products with FP32
  metrics and coefficients add a few ulps.  The test states and media are smooth
  or bounded so that no catastrophic cancellation occurs.
"""
import math

import numpy as np
import pytest
import torch

from oracle import rk
from oracle.elastic import Scheme, rhs
from oracle.metrics import metrics
from oracle.pointwise import PointOracle
from oracle.solver import OracleSolver
from oracle.source import PointSource, moment_tensor
from workloads.configs import config_by_name
from workloads.fields import gaussian_pulse, random_state, smooth_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium
from workloads.timestep import stable_dt

pytestmark = pytest.mark.gpu

MIXED = [("char", 0.0), ("char", 0.3), ("char", -0.4), ("char", 1.0), ("char", 0.0), ("free",)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _problem(nodes, order, geometry="curvy", ext=(1000.0, 1100.0, 900.0), medium="smooth_gradient"):
    X = node_coordinates(make_map(geometry, ext), nodes)
    mat = make_medium(medium, Lz=ext[2])(*X)
    J, a = metrics(*X, order)
    return X, mat, J, a, Scheme(order, nodes)


def _solver(nodes, order, prec, bc, X, mat, keep=False):
    from paper_2011_02600_gb300 import ElasticSolver
    s = ElasticSolver(nodes, order, prec, bc)
    s.setup(torch.from_numpy(np.stack(X)), torch.from_numpy(np.stack(mat)), keep_metrics=keep)
    return s


def _relerr(got, want):
    got = np.asarray(got, dtype=float)
    axes = tuple(range(1, want.ndim))
    return (np.abs(got - want).max(axis=axes) / np.maximum(np.abs(want).max(axis=axes), 1e-300)).max()


SIZES = {2: [(6, 6, 6), (35, 13, 11)], 4: [(11, 11, 11), (37, 19, 14)], 6: [(16, 16, 16), (41, 29, 23)]}


@pytest.mark.parametrize("order", [2, 4, 6])
def test_metrics_fp64(order):
    nodes = SIZES[order][1]
    X, mat, J, a, _ = _problem(nodes, order)
    s = _solver(nodes, order, 64, MIXED, X, mat, keep=True)
    Jg, ag = s.metrics()
    assert np.abs(Jg.cpu().numpy() - J).max() / np.abs(J).max() < 1e-13
    A = np.stack([np.stack(r) for r in a])
    assert np.abs(ag.cpu().numpy() - A).max() / np.abs(A).max() < 1e-13


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 5e-5)])
def test_rhs_parity(order, which, prec, tol):
    nodes = SIZES[order][which]
    X, mat, J, a, sch = _problem(nodes, order)
    s = _solver(nodes, order, prec, MIXED, X, mat)
    if prec == 64:
        Q = random_state(nodes, 100 + order, 1.0, 1.0e6)
    else:
        Q = np.stack(smooth_state(nodes, 5, *_idx(nodes)))
    want = rhs(Q, sch, J, a, mat, MIXED)
    got = s.rhs(torch.from_numpy(Q)).cpu().numpy()
    assert _relerr(got, want) < tol


def _idx(nodes):
    K, Jj, I = np.meshgrid(np.arange(nodes[2]), np.arange(nodes[1]), np.arange(nodes[0]), indexing="ij")
    return I, Jj, K


@pytest.mark.parametrize("order", [4, 6])
def test_all_free_surface_energy_rate_gpu(order):
    """Theorem (free-surface procedure) holds for the GPU right-hand side too:
    <Q, P~^-1 dQ/dt>_H = 0, evaluated with the oracle's H, J and P from the GPU's dQ/dt."""
    nodes = SIZES[order][1]
    X, mat, J, a, sch = _problem(nodes, order)
    free = [("free",)] * 6
    s = _solver(nodes, order, 64, free, X, mat)
    Q = random_state(nodes, 7, 1.0, 1.0)
    d = s.rhs(torch.from_numpy(Q)).cpu().numpy()
    rho, lam, mu = mat
    # P~^-1 dQ/dt: velocity rows rho J dv; stress rows J S dsigma
    W = sch.weights3()
    pv = sum(Q[c] * rho * J * d[c] for c in range(3))
    ds = d[3:9]
    tr = ds[0] + ds[1] + ds[2]
    Sd = [(ds[c] - lam / (3 * lam + 2 * mu) * tr) / (2 * mu) for c in range(3)] + [ds[c] / mu for c in range(3, 6)]
    ps = sum(Q[3 + c] * J * Sd[c] for c in range(6))
    val = float(np.sum(W * (pv + ps)))
    scale = float(np.sum(np.abs(W * pv)))
    assert abs(val) < 1e-12 * scale


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("stage", [0, 3])
def test_fused_stage_parity_fp64(order, stage):
    nodes = SIZES[order][1]
    X, mat, J, a, sch = _problem(nodes, order)
    s = _solver(nodes, order, 64, MIXED, X, mat)
    Q = random_state(nodes, 31, 1.0, 1.0e6)
    dQ = random_state(nodes, 32, 0.1, 1.0e5)
    s.set_state(torch.from_numpy(Q), reset_register=False)
    s.view(s.dq, 9).copy_(torch.from_numpy(dQ))
    dt = 2.5e-3
    s.rk_stage(stage, dt)
    L = rhs(Q, sch, J, a, mat, MIXED)
    dq_new = (rk.A[stage] * dQ if stage else 0.0) + dt * L
    q_new = Q + rk.B[stage] * dq_new
    assert _relerr(s.view(s.dq, 9).cpu().numpy(), dq_new) < 1e-12
    assert _relerr(s.state().cpu().numpy(), q_new) < 1e-12


@pytest.mark.parametrize("order,nodes", [(6, (101, 45, 40)), (4, (70, 33, 30)), (2, (67, 20, 13)),
                                         (6, (16, 16, 16)), (4, (11, 11, 11)), (2, (6, 6, 6)),
                                         (6, (65, 24, 17)), (4, (36, 12, 97)), (6, (37, 16, 200))])
@pytest.mark.parametrize("prec", [32, 64])
def test_tiled_matches_general_kernel(order, nodes, prec):
    """The tiled kernel (several tiles, ragged last tiles, closure rows split across tiles,
    minimum sizes, several s chunks) and the general kernel compute the same right-hand
    side over every node; also checked against the oracle."""
    X, mat, J, a, sch = _problem(nodes, order)
    s = _solver(nodes, order, prec, MIXED, X, mat)
    Q = np.stack(smooth_state(nodes, 9, *_idx(nodes))) if prec == 32 else random_state(nodes, 9)
    r_tiled = s.rhs(torch.from_numpy(Q)).cpu().numpy()
    s.set_kernel_path(1)
    r_gen = s.rhs(torch.from_numpy(Q)).cpu().numpy()
    tol = 1e-12 if prec == 64 else 5e-6
    assert _relerr(r_tiled, r_gen) < tol
    want = rhs(Q, sch, J, a, mat, MIXED)
    assert _relerr(r_tiled, want) < (1e-12 if prec == 64 else 5e-5)


def test_deterministic_fp64():
    nodes, order = SIZES[6][1], 6
    X, mat, J, a, sch = _problem(nodes, order)
    s = _solver(nodes, order, 64, MIXED, X, mat)
    Q = torch.from_numpy(random_state(nodes, 3))
    r1 = s.rhs(Q).clone()
    r2 = s.rhs(Q).clone()
    assert torch.equal(r1, r2)


def test_cube33_order4_run_against_oracle():
    """Workload 1 (33^3, identity map, order 4, FP64, CFL 0.5, 100 steps): energy history and
    four receivers against the oracle."""
    cfg = config_by_name("cube33_o4_fp64")
    nodes, order = cfg.nodes, cfg.order
    fmap = make_map(cfg)
    X = node_coordinates(fmap, nodes)
    mat = make_medium(cfg)(*X)
    dt = stable_dt(*X, *mat, cfg.cfl)
    Q0 = np.stack(gaussian_pulse(*X, (500.0, 500.0, -500.0), cfg.extra["pulse_width"]))
    rec = [(16, 16, 32), (8, 24, 32), (24, 8, 32), (16, 16, 16)]
    orc = OracleSolver(order, *X, mat, cfg.bc)
    orc.Q[:] = Q0
    orc.receivers = rec
    E_or = [orc.energy()]
    orc.step(dt, cfg.steps, E_or)
    s = _solver(nodes, order, 64, cfg.bc, X, mat)
    s.set_state(torch.from_numpy(Q0))
    tr = s.set_receivers(rec, cfg.steps)
    E_gpu = [s.energy()]
    for _ in range(cfg.steps):
        s.step(1, dt)
        E_gpu.append(s.energy())
    E_or, E_gpu = np.array(E_or), np.array(E_gpu)
    assert np.abs(E_gpu - E_or).max() / E_or[0] < 1e-12
    assert np.all(np.diff(E_gpu) <= 1e-13 * E_gpu[0])
    want = np.stack(orc.traces, axis=-1)        # [rec][3][step]
    got = tr.cpu().numpy()
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-11
    assert _relerr(s.state().cpu().numpy(), orc.Q) < 1e-11


def test_source_run_against_oracle():
    """Moment-tensor source (Ricker) on a curvilinear order-6 grid, FP64, 30 steps."""
    nodes, order = (29, 27, 25), 6
    ext = (2000.0, 2000.0, 1500.0)
    X, mat, J, a, sch = _problem(nodes, order, ext=ext)
    bc = [("char", 0.0)] * 5 + [("free",)]
    dt = stable_dt(*X, *mat, 0.5)
    Mv = moment_tensor(0.3, 1.1, -0.7, 1.0e13)
    ref = (0.43, 0.52, 0.61)
    f0 = 25.0
    orc = OracleSolver(order, *X, mat, bc)
    orc.sources.append(PointSource(ref, Mv, lambda t: math.exp(0) * _ricker(t, f0, 1.2 / f0), order, nodes,
                                   sch.weights3(), J))
    orc.step(dt, 30)
    s = _solver(nodes, order, 64, bc, X, mat, keep=True)
    s.set_source(ref, Mv, "ricker", f0=f0)
    s.step(30, dt)
    assert _relerr(s.state().cpu().numpy(), orc.Q) < 1e-11


def _ricker(t, f0, t0):
    a = (math.pi * f0 * (t - t0)) ** 2
    return (1 - 2 * a) * math.exp(-a)


def test_fp32_run_error_vs_fp64_oracle():
    """FP32 error against the FP64 oracle over 50 steps of a pulse on a curvilinear grid
    (order 6), relative to the peak amplitude: the stated FP32 target is 1e-4."""
    nodes, order = (41, 29, 23), 6
    X, mat, J, a, sch = _problem(nodes, order, ext=(4000.0, 2800.0, 2200.0))
    bc = [("char", 0.0)] * 5 + [("free",)]
    dt = stable_dt(*X, *mat, 0.5)
    Q0 = np.stack(gaussian_pulse(*X, (2000.0, 1400.0, 1100.0), 250.0))
    orc = OracleSolver(order, *X, mat, bc)
    orc.Q[:] = Q0
    orc.step(dt, 50)
    s = _solver(nodes, order, 32, bc, X, mat)
    s.set_state(torch.from_numpy(Q0))
    s.step(50, dt)
    got = s.state().cpu().numpy().astype(float)
    err = np.abs(got[:3] - orc.Q[:3]).max() / np.abs(orc.Q[:3]).max()
    assert err < 1e-4, err


def test_full_size_topography_stage_sampled():
    """The bench workload's full size (1025 x 1025 x 401, order 6, FP32, sinusoid
    topography, von Karman medium) in the bench's launch configuration: one fused stage,
    checked at sampled nodes (faces, edges, corners, closure rows, interior) against
    the pointwise oracle."""
    cfg = config_by_name("topo1025_o6_fp32")
    nodes, order = cfg.nodes, cfg.order
    from paper_2011_02600_gb300.workload_setup import build_solver
    s = build_solver(cfg, precision=32)[0]
    fmap = make_map(cfg)
    fmed = make_medium(cfg)
    dev = s.device
    nq, nr, ns = nodes

    def on_gpu_state(seed, scale_v, scale_s):
        out = []
        i = torch.arange(nq, device=dev, dtype=torch.float64).view(1, 1, nq)
        j = torch.arange(nr, device=dev, dtype=torch.float64).view(1, nr, 1)
        k = torch.arange(ns, device=dev, dtype=torch.float64).view(ns, 1, 1)
        return smooth_state(nodes, seed, i, j, k, xp=torch, scale_v=scale_v, scale_s=scale_s)
    st = s.state()
    for f, val in enumerate(on_gpu_state(11, 1.0, 1.0e6)):
        st[f].copy_(val.expand(ns, nr, nq))
    dqv = s.view(s.dq, 9)
    for f, val in enumerate(on_gpu_state(12, 0.1, 1.0e5)):
        dqv[f].copy_(val.expand(ns, nr, nq))
    dt, stage = 2.0e-3, 2
    s.rk_stage(stage, dt)
    torch.cuda.synchronize()
    qn, dqn = s.state(), s.view(s.dq, 9)
    po = PointOracle(order, nodes, fmap, fmed, cfg.bc)

    def fs(i, j, k):
        return smooth_state(nodes, 11, np.asarray(i), np.asarray(j), np.asarray(k))

    def fd(i, j, k):
        return smooth_state(nodes, 12, np.asarray(i), np.asarray(j), np.asarray(k), scale_v=0.1, scale_s=1.0e5)
    rng = np.random.default_rng(0)
    samples = [(0, 0, 0), (nq - 1, nr - 1, ns - 1), (0, nr - 1, ns - 1), (5, 3, ns - 1), (512, 700, ns - 1),
               (512, 512, 200), (6, 6, 6), (nq - 7, 600, 300), (300, nr - 6, 5), (1, 1000, 399)]
    samples += [tuple(int(rng.integers(0, n)) for n in nodes) for _ in range(20)]
    want_q, want_dq, got_q, got_dq = [], [], [], []
    for node in samples:
        wq, wd = po.rk_stage_at(node, stage, dt, fs, fd)
        i, j, k = node
        want_q.append(wq)
        want_dq.append(wd)
        got_q.append(qn[:, k, j, i].double().cpu().numpy())
        got_dq.append(dqn[:, k, j, i].double().cpu().numpy())
    for got, want in ((got_q, want_q), (got_dq, want_dq)):
        got, want = np.array(got), np.array(want)          # [sample][field]
        scale = np.abs(want).max(axis=0)
        err = (np.abs(got - want) / scale).max(axis=0)
        assert np.all(err < 5e-5), (err, samples[int(np.argmax(np.abs(got - want).max(axis=1)))])


def test_batched_solver_matches_single_runs():
    """Batched solver: B states with their own sources, one launch per kernel; every member
    equals its own unbatched run bit for bit (FP32 and FP64)."""
    from paper_2011_02600_gb300 import ElasticSolver
    nodes, order = (41, 37, 30), 4
    X, mat, J, a, sch = _problem(nodes, order, ext=(3000.0, 2800.0, 2200.0))
    bc = [("char", 0.0)] * 5 + [("free",)]
    dt = stable_dt(*X, *mat, 0.5)
    srcs = [dict(ref=(0.4, 0.5, 0.6), moment=list(moment_tensor(0.1, 1.0, 0.2, 1e12))),
            dict(ref=(0.55, 0.35, 0.7), moment=list(moment_tensor(1.1, 0.7, -0.5, 3e12))),
            dict(ref=(0.62, 0.61, 0.45), moment=list(moment_tensor(2.3, 1.3, 1.5, 2e12)))]
    rec = [(10, 10, nodes[2] - 1), (30, 20, nodes[2] - 1)]
    for prec in (32, 64):
        sb = ElasticSolver(nodes, order, prec, bc, batch=3)
        sb.setup(torch.from_numpy(np.stack(X)), torch.from_numpy(np.stack(mat)), keep_metrics=True)
        sb.set_sources(srcs, f0=8.0)
        trb = sb.set_receivers(rec, 40)
        sb.step(40, dt)
        for m, sc in enumerate(srcs):
            s1 = _solver(nodes, order, prec, bc, X, mat, keep=True)
            s1.set_sources([sc], f0=8.0)
            tr1 = s1.set_receivers(rec, 40)
            s1.step(40, dt)
            assert torch.equal(sb.state(m), s1.state())
            assert torch.equal(trb[m], tr1)
