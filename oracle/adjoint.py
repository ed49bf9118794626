"""Receiver misfit of the oracle solver and its derivatives, for checking adjoints (oracle).

Test infrastructure only; see ``oracle/__init__.py``.

The paper has no adjoint; what is checked here is the definition of a
derivative.  The misfit of a run is

    Phi(m) = sum_n  1/2 dt  sum_r |v(x_r, t_{n+1}) - d_r,n|^2,

v recorded after every Runge-Kutta step (the oracle's scheme, Sections 4-5,
with the material m = (rho, lambda, mu) per node).  Its directional derivative
is taken by the complex step Im Phi(m + i h dm) / h, which has no cancellation
error, and by central differences.  ``assemble_operator`` builds the matrix of
the semi-discrete operator column by column so that its transpose is explicit.
"""
import numpy as np

from . import rk
from .elastic import Scheme, rhs
from .metrics import metrics


def misfit(order, X, mat, bc, receivers, data, dt, nsteps, source=None, Q0=None):
    """Phi for material mat = (rho, lam, mu) (real or complex arrays).

    receivers: list of (i, j, k); data: array [nsteps][n_rec][3]; source: callable
    (dQdt, t) -> None adding the source term (optional); Q0: initial state.
    """
    nodes = (X[0].shape[2], X[0].shape[1], X[0].shape[0])
    J, a = metrics(*X, order)
    sch = Scheme(order, nodes)
    dtype = np.result_type(*[np.asarray(m) for m in mat])
    Q = np.zeros((9,) + J.shape, dtype=dtype)
    if Q0 is not None:
        Q += Q0
    dQ = np.zeros_like(Q)

    def L(q, t):
        d = rhs(q, sch, J, a, mat, bc)
        if source is not None:
            source(d, t)
        return d
    phi = 0.0
    for n in range(nsteps):
        rk.rk_step(Q, dQ, n * dt, dt, L)
        for r, (i, j, k) in enumerate(receivers):
            for c in range(3):
                diff = Q[c][k, j, i] - data[n][r][c]
                phi = phi + 0.5 * dt * diff * diff
    return phi


def complex_step(order, X, mat, dmat, bc, receivers, data, dt, nsteps, source=None, h=1e-30):
    """Directional derivative dPhi/dm . dm by the complex step."""
    mc = tuple(np.asarray(m, dtype=complex) + 1j * h * np.asarray(dm) for m, dm in zip(mat, dmat))
    return float(np.imag(misfit(order, X, mc, bc, receivers, data, dt, nsteps, source)) / h)


def assemble_operator(order, X, mat, bc):
    """Dense matrix of Q -> dQ/dt (9 fields flattened in [field][s][r][q] order)."""
    nodes = (X[0].shape[2], X[0].shape[1], X[0].shape[0])
    J, a = metrics(*X, order)
    sch = Scheme(order, nodes)
    n = 9 * J.size
    Lm = np.zeros((n, n))
    e = np.zeros(n)
    for col in range(n):
        e[:] = 0.0
        e[col] = 1.0
        Lm[:, col] = rhs(e.reshape((9,) + J.shape), sch, J, a, mat, bc).ravel()
    return Lm
