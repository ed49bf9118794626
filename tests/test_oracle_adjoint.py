"""Pins of the oracle's derivative tools used to check the adjoint."""
import numpy as np

from oracle.adjoint import assemble_operator, misfit
from oracle.elastic import Scheme
from oracle.metrics import metrics
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium


def _setup(order=2, nodes=(7, 6, 6)):
    X = node_coordinates(make_map("curvy", (1.0, 1.1, 0.9)), nodes)
    rng = np.random.default_rng(2)
    shape = X[0].shape
    mat = (rng.uniform(1.0, 2.0, shape), rng.uniform(0.5, 1.5, shape), rng.uniform(0.5, 1.5, shape))
    return X, mat


def test_complex_step_matches_central_difference():
    X, mat = _setup()
    bc = [("char", 0.0), ("free",), ("char", 0.4), ("free",), ("char", -0.3), ("free",)]
    rec = [(3, 2, 5), (1, 4, 5)]
    rng = np.random.default_rng(3)
    data = rng.normal(size=(6, 2, 3))
    Q0 = rng.normal(size=(9,) + X[0].shape)
    dm = tuple(rng.normal(size=X[0].shape) for _ in range(3))
    dt = 0.01
    src = None
    from oracle import adjoint as oa
    cs = np.imag(oa.misfit(2, X, tuple(np.asarray(m, complex) + 1e-30j * d for m, d in zip(mat, dm)), bc, rec, data,
                           dt, 6, src, Q0=Q0)) / 1e-30
    h = 1e-6
    fp = misfit(2, X, tuple(m + h * d for m, d in zip(mat, dm)), bc, rec, data, dt, 6, src, Q0=Q0)
    fm = misfit(2, X, tuple(m - h * d for m, d in zip(mat, dm)), bc, rec, data, dt, 6, src, Q0=Q0)
    fd = (fp - fm) / (2 * h)
    assert abs(cs - fd) < 1e-6 * abs(cs)


def test_assembled_operator_is_skew_in_the_energy_inner_product():
    """Free surfaces everywhere: (H P~^-1) L is skew-symmetric (the free-surface energy theorem
    as a matrix identity), which pins the column-by-column assembly."""
    X, mat = _setup()
    nodes = (X[0].shape[2], X[0].shape[1], X[0].shape[0])
    Lm = assemble_operator(2, X, mat, [("free",)] * 6)
    J, _ = metrics(*X, 2)
    W = Scheme(2, nodes).weights3().ravel()
    rho, lam, mu = (m.ravel() for m in mat)
    Jr = J.ravel()
    n = Jr.size
    Pinv = np.zeros((9 * n, 9 * n))
    for c in range(3):
        idx = np.arange(c * n, (c + 1) * n)
        Pinv[idx, idx] = W * rho * Jr
    # stress block: J S per node (S = C^-1, engineering shear)
    for p in range(n):
        C = np.zeros((6, 6))
        C[:3, :3] = lam[p]
        C[np.arange(3), np.arange(3)] += 2 * mu[p]
        C[3, 3] = C[4, 4] = C[5, 5] = mu[p]
        S = np.linalg.inv(C) * Jr[p] * W[p]
        idx = np.array([(3 + c) * n + p for c in range(6)])
        Pinv[np.ix_(idx, idx)] = S
    A = Pinv @ Lm
    assert np.abs(A + A.T).max() < 1e-11 * np.abs(A).max()


def test_misfit_quadrature_closed_forms():
    """Phi = sum_n 1/2 dt sum_r |v(x_r, t_{n+1}) - d_{r,n}|^2: with a zero state (no source)
    it is 1/2 dt times the data's squared sum; with the solver's own traces as data it is 0."""
    from oracle.solver import OracleSolver
    from workloads.fields import random_state
    nodes, order = (9, 8, 7), 2
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    bc = [("char", 0.0)] * 5 + [("free",)]
    rec = [(2, 3, 6), (5, 4, 3)]
    dt, nsteps = 1e-3, 5
    rng = np.random.default_rng(3)
    data = rng.normal(size=(nsteps, len(rec), 3))
    phi0 = misfit(order, X, mat, bc, rec, data, dt, nsteps)
    assert abs(phi0 - 0.5 * dt * float(np.sum(data ** 2))) < 1e-14 * phi0
    Q0 = random_state(nodes, 5, 1.0, 1.0e6)
    orc = OracleSolver(order, *X, mat, bc)
    orc.Q[:] = Q0
    orc.receivers = rec
    orc.step(dt, nsteps)
    own = np.array(orc.traces)
    assert misfit(order, X, mat, bc, rec, own, dt, nsteps, Q0=Q0) < 1e-24 * float(np.sum(own ** 2))
