"""The general adjoint kernels' per-node bodies on the CPU: tests/host_adjoint.cpp compiles
adjoint_prep_at and adjoint_stage_at (csrc/adjoint_node.cuh: L^T with the transposed face terms,
the adjoint Runge-Kutta updates and the material gradient, with their division-free factors)
as host C++ and runs them over every node, FP64.  Against the oracle:

* L^T equals the transpose of the oracle's assembled operator on a tiny grid, and satisfies
  <L x, y> = <x, L^T y> with the oracle's L on larger grids, orders 2 to 7, every face kind;
* one adjoint stage updates Ub and Wb as the exact adjoint of the 2N-storage stage prescribes;
* its material gradient equals dt <Wb_k, d(L U)/dm . dm> with the derivative of the oracle's
  right-hand side taken by the complex step (no cancellation error)."""
import ctypes

import numpy as np
import pytest

from oracle import rk
from oracle.adjoint import assemble_operator
from oracle.elastic import Scheme, rhs
from oracle.metrics import metrics
from workloads.fields import random_state
from workloads.geometry import make_map, node_coordinates

from host_build import build

BCS = {
    "free": [("free",)] * 6,
    "char": [("char", g) for g in (0.0, 0.3, -0.4, 1.0, -1.0, 0.25)],
    "mixed": [("char", 0.0), ("free",), ("char", 0.6), ("free",), ("char", -0.2), ("free",)],
}


@pytest.fixture(scope="module")
def hostadj(tmp_path_factory):
    so = build("host_adjoint.cpp", tmp_path_factory.mktemp("hostadj") / "libhostadj.so", shared=True)
    lib = ctypes.CDLL(so)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.host_rhs_adjoint.argtypes = [I] * 4 + [P] * 7
    lib.host_adjoint_stage.argtypes = [I] * 4 + [D] * 3 + [P] * 10
    lib.host_rhs_adjoint.restype = lib.host_adjoint_stage.restype = I
    return lib


def _problem(order, nodes, seed):
    X = node_coordinates(make_map("curvy", (1.0, 1.1, 0.9)), nodes)
    J, a = metrics(*X, order)
    rng = np.random.default_rng(seed)
    mat = (rng.uniform(1.0, 2.0, J.shape), rng.uniform(0.5, 1.5, J.shape), rng.uniform(0.5, 1.5, J.shape))
    return X, J, a, mat


def _arrays(J, a, mat):
    rho, lam, mu = mat
    met = np.ascontiguousarray(np.stack([a[xi][c] for xi in range(3) for c in range(3)]))
    coef = np.ascontiguousarray(np.stack([1.0 / (rho * J), lam / J, mu / J]))
    rlmj = np.ascontiguousarray(np.stack([rho, lam, mu, J]))
    return met, coef, rlmj


def _bc(bc):
    kind = (ctypes.c_int * 6)(*[0 if b[0] == "free" else 1 for b in bc])
    gamma = (ctypes.c_double * 6)(*[0.0 if b[0] == "free" else b[1] for b in bc])
    return ctypes.cast(kind, ctypes.c_void_p), ctypes.cast(gamma, ctypes.c_void_p), (kind, gamma)


def _LT(lib, order, J, a, mat, bc, w):
    ns, nr, nq = J.shape
    met, coef, _ = _arrays(J, a, mat)
    kind, gamma, keep = _bc(bc)
    w = np.ascontiguousarray(w, dtype=np.float64)
    scratch = np.zeros_like(w)
    out = np.zeros_like(w)
    assert lib.host_rhs_adjoint(order, nq, nr, ns, w.ctypes.data, met.ctypes.data, coef.ctypes.data, kind, gamma,
                                scratch.ctypes.data, out.ctypes.data) == 0
    return out


@pytest.mark.parametrize("bcname", sorted(BCS))
def test_transpose_full_matrix_tiny_grid(hostadj, bcname):
    order, nodes = 2, (6, 7, 6)
    X, J, a, mat = _problem(order, nodes, 1)
    Lm = assemble_operator(order, X, mat, BCS[bcname])
    n = Lm.shape[0]
    LT = np.zeros_like(Lm)
    e = np.zeros(n)
    for col in range(n):
        e[:] = 0.0
        e[col] = 1.0
        LT[:, col] = _LT(hostadj, order, J, a, mat, BCS[bcname], e.reshape((9,) + J.shape)).ravel()
    assert np.abs(LT - Lm.T).max() < 1e-12 * np.abs(Lm).max()


@pytest.mark.parametrize("order,nodes", [(2, (12, 9, 8)), (3, (9, 8, 10)), (4, (14, 12, 11)), (5, (13, 12, 14)),
                                         (6, (19, 17, 16)), (7, (17, 16, 18))])
@pytest.mark.parametrize("bcname", sorted(BCS))
def test_transpose_dot_product(hostadj, order, nodes, bcname):
    X, J, a, mat = _problem(order, nodes, 2)
    bc = BCS[bcname]
    sch = Scheme(order, nodes)
    for seed in range(2):
        x = random_state(nodes, 40 + seed, 1.0, 1.0)
        y = random_state(nodes, 50 + seed, 1.0, 1.0)
        Lx = rhs(x, sch, J, a, mat, bc)
        LTy = _LT(hostadj, order, J, a, mat, bc, y)
        lhs, rhs_ = float(np.sum(Lx * y)), float(np.sum(x * LTy))
        scale = float(np.sum(np.abs(Lx * y)))
        assert abs(lhs - rhs_) < 1e-12 * scale, (lhs, rhs_, scale)


@pytest.mark.parametrize("order,nodes", [(2, (9, 8, 7)), (3, (8, 9, 7)), (4, (13, 12, 11)), (5, (12, 11, 13)),
                                         (6, (17, 16, 18)), (7, (16, 18, 17))])
@pytest.mark.parametrize("bcname", ["char", "mixed"])
def test_adjoint_stage_updates_and_gradient(hostadj, order, nodes, bcname):
    X, J, a, mat = _problem(order, nodes, 3)
    bc = BCS[bcname]
    ns, nr, nq = J.shape
    met, coef, rlmj = _arrays(J, a, mat)
    kind, gamma, keep = _bc(bc)
    k, dt = 2, 1.0e-3
    A, Bk = float(rk.A[k]), float(rk.B[k])
    U = random_state(nodes, 60, 1.0, 1.0)
    U0 = random_state(nodes, 61, 1.0, 1.0)
    W0 = random_state(nodes, 62, 1.0, 1.0)
    ubar, wbar = U0.copy(), W0.copy()
    scratch = np.zeros_like(U)
    grad = np.zeros((3,) + J.shape)
    assert hostadj.host_adjoint_stage(order, nq, nr, ns, A, Bk, dt, U.ctypes.data, ubar.ctypes.data,
                                      wbar.ctypes.data, scratch.ctypes.data, met.ctypes.data, coef.ctypes.data,
                                      rlmj.ctypes.data, kind, gamma, grad.ctypes.data) == 0
    # Wb_k = Wb + B_k Ub_{k+1};  Ub_k = Ub_{k+1} + dt L^T Wb_k;  Wb <- A_k Wb_k
    Wk = W0 + Bk * U0
    sc = np.abs(U0).max()
    assert np.abs(ubar - (U0 + dt * _LT(hostadj, order, J, a, mat, bc, Wk))).max() < 1e-13 * sc
    assert np.abs(wbar - A * Wk).max() < 1e-14 * np.abs(Wk).max()
    # gradient: dt <Wb_k, (d(L U)/dm) dm> by the complex step on the oracle's L
    sch = Scheme(order, nodes)
    rng = np.random.default_rng(7)
    h = 1e-30
    for _ in range(3):
        dm = [rng.normal(size=J.shape) * m for m in mat]
        matc = tuple(np.asarray(m, complex) + 1j * h * d for m, d in zip(mat, dm))
        dLU = np.imag(rhs(U.astype(complex), sch, J, a, matc, bc)) / h
        want = dt * float(np.sum(Wk * dLU))
        got = float(sum(np.sum(grad[f] * dm[f]) for f in range(3)))
        assert abs(got - want) < 1e-11 * abs(want), (got, want)


@pytest.mark.parametrize("order,nodes", [(2, (7, 6, 8)), (4, (12, 11, 13)), (6, (16, 17, 18))])
@pytest.mark.parametrize("bcname", sorted(BCS))
def test_traditional_transpose_dot_product(hostadj, order, nodes, bcname):
    """The adjoint bodies with the traditional operators (OpCoef<kTraditional + order>) satisfy
    <L x, y> = <x, L^T y> with the oracle's traditional scheme."""
    from paper_2011_02600_gb300.opgen import TRADITIONAL
    X, J, a, mat = _problem(order, nodes, 4)
    bc = BCS[bcname]
    sch = Scheme(order, nodes, "traditional")
    x = random_state(nodes, 70, 1.0, 1.0)
    y = random_state(nodes, 71, 1.0, 1.0)
    Lx = rhs(x, sch, J, a, mat, bc)
    LTy = _LT(hostadj, TRADITIONAL + order, J, a, mat, bc, y)
    lhs, rhs_ = float(np.sum(Lx * y)), float(np.sum(x * LTy))
    assert abs(lhs - rhs_) < 1e-12 * float(np.sum(np.abs(Lx * y))), (lhs, rhs_)
