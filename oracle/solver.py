"""Time loop of the oracle: RK4 over the semi-discrete scheme, receivers, energy.

Test infrastructure only; see ``oracle/__init__.py``.
"""
import numpy as np

from . import rk
from .elastic import Scheme, energy, rhs
from .metrics import metrics


class OracleSolver:
    """Plain FP64 solver on one curvilinear block.

    x, y, z: node coordinates [s][r][q]; mat: (rho, lam, mu) arrays; bc: six
    face conditions (q0, q1, r0, r1, s0, s1); operator: "upwind" (Table 1) or
    "traditional" (Table 2), as in elastic.Scheme.  The metric terms use the upwind pair's
    D_c of the same order either way.
    """

    def __init__(self, order, x, y, z, mat, bc, operator="upwind"):
        self.nodes = (x.shape[2], x.shape[1], x.shape[0])
        self.order = order
        self.scheme = Scheme(order, self.nodes, operator)
        self.J, self.a = metrics(x, y, z, order)
        self.mat = tuple(np.asarray(m, dtype=float) for m in mat)
        self.bc = list(bc)
        self.Q = np.zeros((9,) + self.J.shape)
        self.dQ = np.zeros_like(self.Q)
        self.t = 0.0
        self.sources = []
        self.receivers = []     # (i, j, k) node indices
        self.traces = []

    def L(self, Q, t):
        d = rhs(Q, self.scheme, self.J, self.a, self.mat, self.bc)
        for s in self.sources:
            s.add_to(d, t)
        return d

    def energy(self):
        return energy(self.Q, self.scheme, self.J, self.mat)

    def record(self):
        if self.receivers:
            self.traces.append(np.array([[self.Q[c][k, j, i] for c in range(3)]
                                         for (i, j, k) in self.receivers]))

    def step(self, dt, n=1, energies=None):
        for _ in range(n):
            rk.rk_step(self.Q, self.dQ, self.t, dt, self.L)
            self.t += dt
            self.record()
            if energies is not None:
                energies.append(self.energy())
        return self
