"""The hand-written adjoint (sbp_rhs_adjoint, sbp_adjoint_stage) and the material gradient.

* L^T against the oracle's L: dot-product tests <L x, y> = <x, L^T y> on several grids,
  orders and boundary mixes, and the full matrix on a tiny grid (exact to rounding, FP64).
* The gradient of the receiver misfit (FP64 path) against the oracle's complex-step
  directional derivatives (no cancellation error) and against central finite
  differences in 20 seeded directions (target: 1e-5 relative).
* sqrt(N) checkpointing does not change the gradient; the autograd.Function returns it.
"""
import numpy as np
import pytest
import torch

from oracle.adjoint import assemble_operator, complex_step
from oracle.elastic import Scheme, rhs
from oracle.metrics import metrics
from oracle.source import PointSource, moment_tensor, ricker
from workloads.fields import random_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium
from workloads.timestep import stable_dt

pytestmark = pytest.mark.gpu

MIXED = [("char", 0.0), ("char", 0.3), ("char", -0.4), ("char", 1.0), ("char", 0.0), ("free",)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _solver(nodes, order, prec, bc, X, mat, keep=False):
    from paper_2011_02600_gb300 import ElasticSolver
    s = ElasticSolver(nodes, order, prec, bc)
    s.setup(torch.from_numpy(np.stack(X)), torch.from_numpy(np.stack(mat)), keep_metrics=keep)
    return s


def _gpu_LT(s, y):
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    w = s.to_layout(torch.from_numpy(y), s.dtype)
    out = s.new_fields(9)
    scratch = s.new_fields(9)
    L.sbp_rhs_adjoint(s.h, w, out, scratch, _stream())
    return s.view(out, 9).cpu().numpy()


@pytest.mark.parametrize("order,nodes", [(2, (12, 9, 8)), (4, (14, 12, 11)), (6, (19, 17, 16))])
@pytest.mark.parametrize("bc", ["mixed", "free"])
def test_transpose_dot_product(order, nodes, bc):
    bcs = MIXED if bc == "mixed" else [("free",)] * 6
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    J, a = metrics(*X, order)
    s = _solver(nodes, order, 64, bcs, X, mat)
    for seed in range(3):
        x = random_state(nodes, 40 + seed, 1.0, 1.0e6)
        y = random_state(nodes, 50 + seed, 1.0e-6, 1.0)
        Lx = rhs(x, Scheme(order, nodes), J, a, mat, bcs)
        LTy = _gpu_LT(s, y)
        lhs, rhs_ = float(np.sum(Lx * y)), float(np.sum(x * LTy))
        scale = float(np.sum(np.abs(Lx * y)))
        assert abs(lhs - rhs_) < 1e-12 * scale, (lhs, rhs_, scale)


def test_transpose_full_matrix_tiny_grid():
    nodes, order = (6, 7, 6), 2
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    Lm = assemble_operator(order, X, mat, MIXED)
    s = _solver(nodes, order, 64, MIXED, X, mat)
    n = Lm.shape[0]
    LT = np.zeros_like(Lm)
    e = np.zeros(n)
    for col in range(n):
        e[:] = 0.0
        e[col] = 1.0
        LT[:, col] = _gpu_LT(s, e.reshape((9,) + X[0].shape)).ravel()
    assert np.abs(LT - Lm.T).max() < 1e-12 * np.abs(Lm).max()


def _misfit_case(nsteps=30, order=4, nodes=(15, 14, 13)):
    ext = (1000.0, 1100.0, 900.0)
    X = node_coordinates(make_map("curvy", ext), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    bc = [("char", 0.0), ("char", 0.0), ("char", 0.2), ("char", 0.0), ("char", -0.3), ("free",)]
    dt = stable_dt(*X, *mat, 0.4)
    rec = [(3, 3, nodes[2] - 1), (10, 4, nodes[2] - 1), (7, 9, nodes[2] - 1), (5, 6, nodes[2] - 3)]
    rng = np.random.default_rng(11)
    data = rng.normal(scale=1e-4, size=(len(rec), 3, nsteps))
    Mv = moment_tensor(0.4, 1.0, 0.3, 1.0e12)
    f0 = 20.0
    src = dict(ref=(0.5, 0.45, 0.55), moment=list(Mv), stf="ricker", f0=f0)
    return dict(X=X, mat=mat, bc=bc, dt=dt, rec=rec, data=data, Mv=Mv, f0=f0, src=src, nsteps=nsteps, order=order,
                nodes=nodes)


def _gpu_problem(c, prec=64, checkpoint_every=None):
    from paper_2011_02600_gb300.adjoint import MisfitProblem
    s = _solver(c["nodes"], c["order"], prec, c["bc"], c["X"], c["mat"], keep=True)
    p = MisfitProblem(s, c["rec"], torch.from_numpy(c["data"]), c["dt"], c["nsteps"], source=c["src"],
                      checkpoint_every=checkpoint_every)
    return p


def _set(p, mat):
    dev = p.s.device
    p.set_material(*(torch.from_numpy(np.asarray(m)).to(dev) for m in mat))


def _directions(c, count, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(tuple(rng.normal(size=c["X"][0].shape) * np.asarray(m) for m in c["mat"]))
    return out


def test_gradient_against_oracle_complex_step():
    c = _misfit_case()
    p = _gpu_problem(c)
    _set(p, c["mat"])
    phi = p.forward()
    g = p.gradient().cpu().numpy()
    nodes = c["nodes"]
    J, _ = metrics(*c["X"], c["order"])
    W = Scheme(c["order"], nodes).weights3()
    psrc = PointSource(c["src"]["ref"], c["Mv"], lambda t: ricker(t, c["f0"], 1.2 / c["f0"]), c["order"], nodes, W, J)
    data_or = np.transpose(c["data"], (2, 0, 1))
    from oracle.adjoint import misfit
    phi_or = misfit(c["order"], c["X"], c["mat"], c["bc"], c["rec"], data_or, c["dt"], c["nsteps"], psrc.add_to)
    assert abs(phi - phi_or) < 1e-12 * abs(phi_or)
    for dm in _directions(c, 4):
        cs = complex_step(c["order"], c["X"], c["mat"], dm, c["bc"], c["rec"], data_or, c["dt"], c["nsteps"],
                          psrc.add_to)
        got = float(sum(np.sum(g[f] * dm[f]) for f in range(3)))
        assert abs(got - cs) < 1e-9 * abs(cs), (got, cs)


def test_gradient_against_finite_differences_20_directions():
    c = _misfit_case()
    p = _gpu_problem(c)
    _set(p, c["mat"])
    p.forward()
    g = p.gradient().cpu().numpy()
    h = 1e-6
    worst = 0.0
    for dm in _directions(c, 20, seed=5):
        _set(p, tuple(m + h * d for m, d in zip(c["mat"], dm)))
        fp = p.forward()
        _set(p, tuple(m - h * d for m, d in zip(c["mat"], dm)))
        fm = p.forward()
        fd = (fp - fm) / (2 * h)
        got = float(sum(np.sum(g[f] * dm[f]) for f in range(3)))
        worst = max(worst, abs(got - fd) / abs(fd))
    assert worst < 1e-5, worst


def test_checkpointing_does_not_change_the_gradient():
    c = _misfit_case(nsteps=24)
    grads = []
    for C in (1, 5, 24):
        p = _gpu_problem(c, checkpoint_every=C)
        _set(p, c["mat"])
        p.forward()
        grads.append(p.gradient().cpu().numpy())
    assert np.array_equal(grads[0], grads[1]) and np.array_equal(grads[1], grads[2])


def test_autograd_function():
    from paper_2011_02600_gb300.adjoint import ElasticMisfit
    c = _misfit_case(nsteps=12)
    p = _gpu_problem(c)
    dev = p.s.device
    rho, lam, mu = (torch.from_numpy(np.asarray(m)).to(dev).requires_grad_(True) for m in c["mat"])
    phi = ElasticMisfit.apply(rho, lam, mu, p)
    gr = torch.autograd.grad(phi, (rho, lam, mu))
    p2 = _gpu_problem(c)
    _set(p2, c["mat"])
    p2.forward()
    g = p2.gradient()
    for f in range(3):
        assert torch.equal(gr[f], g[f])


@pytest.mark.parametrize("order,nodes", [(2, (40, 20, 13)), (4, (70, 19, 30)), (6, (45, 30, 40)), (4, (11, 11, 11)),
                                         (6, (16, 17, 16))])
@pytest.mark.parametrize("prec", [64, 32])
def test_tiled_adjoint_matches_general_path(order, nodes, prec):
    """The tiled kernel's adjoint passes (L^T on yhat, the gradient on U_k: several tiles,
    ragged and minimum sizes) against the general one-thread-per-node adjoint kernels: L^T y,
    and a whole misfit gradient (forward run, checkpoints, adjoint stages)."""
    ext = (1000.0, 1100.0, 900.0)
    X = node_coordinates(make_map("curvy", ext), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    s = _solver(nodes, order, prec, MIXED, X, mat)
    y = random_state(nodes, 61, 1.0e-6, 1.0)
    LT = []
    for path in (0, 1):
        s.set_kernel_path(path)
        LT.append(_gpu_LT(s, y))
    tol = 1e-12 if prec == 64 else 2e-5
    scale = np.abs(LT[1]).max(axis=(1, 2, 3), keepdims=True)
    assert np.abs(LT[0] - LT[1]).max() < tol * scale.max()
    assert (np.abs(LT[0] - LT[1]) / scale).max() < tol
    c = _misfit_case(nsteps=6, order=order, nodes=nodes)
    c["bc"] = MIXED
    grads = []
    for path in (0, 1):
        p = _gpu_problem(c, prec)
        p.s.set_kernel_path(path)
        _set(p, c["mat"])
        p.forward()
        grads.append(p.gradient().double().cpu().numpy())
    for f in range(3):
        sc = np.abs(grads[1][f]).max()
        assert np.abs(grads[0][f] - grads[1][f]).max() < (1e-11 if prec == 64 else 1e-4) * sc, f


def _batched_problem(c, sources, prec=64, path=0):
    from paper_2011_02600_gb300 import ElasticSolver
    from paper_2011_02600_gb300.adjoint import MisfitProblem
    s = ElasticSolver(c["nodes"], c["order"], prec, c["bc"], batch=len(sources))
    s.setup(torch.from_numpy(np.stack(c["X"])), torch.from_numpy(np.stack(c["mat"])), keep_metrics=True)
    s.set_kernel_path(path)
    rng = np.random.default_rng(21)
    data = rng.normal(scale=1e-4, size=(len(sources), len(c["rec"]), 3, c["nsteps"]))
    return MisfitProblem(s, c["rec"], torch.from_numpy(data), c["dt"], c["nsteps"], sources=sources, f0=c["f0"]), data


def _three_sources():
    return [dict(ref=(0.5, 0.45, 0.55), moment=list(moment_tensor(0.4, 1.0, 0.3, 1.0e12))),
            dict(ref=(0.35, 0.6, 0.7), moment=list(moment_tensor(1.3, 0.6, -0.9, 2.0e12))),
            dict(ref=(0.62, 0.4, 0.45), moment=list(moment_tensor(2.2, 1.2, 1.4, 0.5e12)))]


@pytest.mark.parametrize("path", [0, 1])
def test_batched_adjoint_is_the_sum_of_single_source_gradients(path):
    """Three sources as one batch (one launch per adjoint kernel, every member adding into one
    gradient): the misfit and the gradient equal the sums of the three single-source problems
    (FP64, tiled and general kernels)."""
    from paper_2011_02600_gb300.adjoint import MisfitProblem
    c = _misfit_case(nsteps=20)
    srcs = _three_sources()
    pb, data = _batched_problem(c, srcs, path=path)
    _set(pb, c["mat"])
    phi_b = pb.forward()
    g_b = pb.gradient().cpu().numpy()
    phi_s, g_s = 0.0, 0.0
    for m, sc in enumerate(srcs):
        s = _solver(c["nodes"], c["order"], 64, c["bc"], c["X"], c["mat"], keep=True)
        s.set_kernel_path(path)
        p = MisfitProblem(s, c["rec"], torch.from_numpy(data[m]), c["dt"], c["nsteps"],
                          source=dict(ref=sc["ref"], moment=sc["moment"], stf="ricker", f0=c["f0"]))
        _set(p, c["mat"])
        phi_s += p.forward()
        g_s = g_s + p.gradient().cpu().numpy()
    assert abs(phi_b - phi_s) < 1e-13 * abs(phi_s)
    for f in range(3):
        assert np.abs(g_b[f] - g_s[f]).max() < 1e-12 * np.abs(g_s[f]).max(), f


def test_batched_gradient_against_finite_differences():
    """The batched problem's gradient against central differences of its summed misfit in
    20 seeded directions (FP64, 1e-5)."""
    c = _misfit_case(nsteps=20)
    pb, _ = _batched_problem(c, _three_sources())
    _set(pb, c["mat"])
    pb.forward()
    g = pb.gradient().cpu().numpy()
    h = 1e-6
    worst = 0.0
    for dm in _directions(c, 20, seed=9):
        _set(pb, tuple(m + h * d for m, d in zip(c["mat"], dm)))
        fp = pb.forward()
        _set(pb, tuple(m - h * d for m, d in zip(c["mat"], dm)))
        fm = pb.forward()
        fd = (fp - fm) / (2 * h)
        got = float(sum(np.sum(g[f] * dm[f]) for f in range(3)))
        worst = max(worst, abs(got - fd) / abs(fd))
    assert worst < 1e-5, worst


@pytest.mark.parametrize("order,nodes", [(2, (21, 18, 16)), (4, (40, 19, 30)), (6, (36, 30, 27))])
@pytest.mark.parametrize("prec", [64, 32])
def test_fused_adjoint_step_matches_stage_by_stage(order, nodes, prec):
    """sbp_adjoint_step (each stage's pointwise prep formed in the previous stage's L^T pass)
    against five sbp_adjoint_stage calls per step: the whole misfit gradient, and Ub at the end."""
    c = _misfit_case(nsteps=8, order=order, nodes=nodes)
    grads = []
    for fused in (True, False):
        p = _gpu_problem(c, prec)
        p.fused = fused
        _set(p, c["mat"])
        p.forward()
        grads.append(p.gradient().double().cpu().numpy())
    for f in range(3):
        sc = np.abs(grads[1][f]).max()
        assert sc > 0
        assert np.abs(grads[0][f] - grads[1][f]).max() < (1e-12 if prec == 64 else 1e-5) * sc, f
