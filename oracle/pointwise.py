"""The oracle's scheme evaluated at individual nodes (for sampled parity at full size).

Test infrastructure only; see ``oracle/__init__.py``.

Computes exactly what ``elastic.rhs`` computes, one node at a time, from
closed-form inputs (mesh map, medium, state functions): each derivative is
the node's row of D+- (or D_c for the metric derivatives) applied to the
values on the nodes that row touches.  It exists so that outputs of a
421M-node grid can be checked at sampled nodes without holding the grid on
the host.
"""
import numpy as np

from . import rk
from .elastic import apply_P, face_penalty, flux, strain_rows
from .metrics import jacobian_and_metrics
from .operators import upwind_pair


class PointOracle:
    """fmap(q, r, s) -> (x, y, z); fmed(x, y, z) -> (rho, lam, mu);
    fstate(i, j, k) -> list of 9 arrays (node-index arguments)."""

    def __init__(self, order, nodes, fmap, fmed, bc):
        self.order = order
        self.nodes = tuple(nodes)
        self.fmap = fmap
        self.fmed = fmed
        self.bc = list(bc)
        self.H, self.Dm, self.Dp, self.Dc = [], [], [], []
        for N in self.nodes:
            H, Dm, Dp = upwind_pair(order, N)
            self.H.append(H)
            self.Dm.append(Dm.tocsr())
            self.Dp.append(Dp.tocsr())
            self.Dc.append((0.5 * (Dp + Dm)).tocsr())

    @staticmethod
    def _row(D, i):
        lo, hi = D.indptr[i], D.indptr[i + 1]
        return D.indices[lo:hi], D.data[lo:hi]

    def _shift(self, node, xi, cols):
        """Index arrays of the nodes obtained by replacing axis xi of ``node`` by ``cols``."""
        ijk = [np.full(len(cols), node[0]), np.full(len(cols), node[1]), np.full(len(cols), node[2])]
        ijk[xi] = np.asarray(cols)
        return ijk

    def coords(self, i, j, k):
        nq, nr, ns = self.nodes
        return self.fmap(np.asarray(i) / (nq - 1), np.asarray(j) / (nr - 1), np.asarray(k) / (ns - 1))

    def metrics_at(self, node):
        """(J, a) at one node from D_c rows applied to the map along each axis."""
        d = []
        for xi in range(3):
            cols, vals = self._row(self.Dc[xi], node[xi])
            X = self.coords(*self._shift(node, xi, cols))
            d.append([float(np.dot(vals, np.broadcast_to(c, vals.shape))) for c in X])
        (x_q, y_q, z_q), (x_r, y_r, z_r), (x_s, y_s, z_s) = d
        return jacobian_and_metrics(x_q, x_r, x_s, y_q, y_r, y_s, z_q, z_r, z_s)

    def material_at(self, node):
        x, y, z = self.coords(*node)
        return tuple(float(np.broadcast_to(m, ())) for m in self.fmed(x, y, z))

    def rhs_at(self, node, fstate):
        """dQ/dt (9 values) at one node (i, j, k)."""
        node = tuple(int(v) for v in node)
        J, a = self.metrics_at(node)
        rv = [0.0, 0.0, 0.0]
        e = [0.0] * 6
        for xi in range(3):
            cols, vals = self._row(self.Dm[xi], node[xi])
            idx = self._shift(node, xi, cols)
            S = fstate(*idx)
            sig = [np.broadcast_to(S[3 + c], vals.shape) for c in range(6)]
            axi = [[], [], []]
            for m in range(len(cols)):
                nb = tuple(int(c[m]) for c in idx)
                _, am = self.metrics_at(nb)
                for c in range(3):
                    axi[c].append(am[xi][c])
            F = flux([np.array(c) for c in axi], sig)
            for c in range(3):
                rv[c] += float(np.dot(vals, F[c]))
            cols, vals = self._row(self.Dp[xi], node[xi])
            S = fstate(*self._shift(node, xi, cols))
            dv = [float(np.dot(vals, np.broadcast_to(S[c], vals.shape))) for c in range(3)]
            B = strain_rows(a[xi], dv)
            for c in range(6):
                e[c] += B[c]
        mat = self.material_at(node)
        Q0 = [float(np.broadcast_to(c, ())) for c in fstate(*[np.asarray(v) for v in node])]
        for face in range(6):
            xi, side = divmod(face, 2)
            if node[xi] != (0 if side == 0 else self.nodes[xi] - 1):
                continue
            out = face_penalty(Q0[0:3], Q0[3:9], a[xi], *mat, side, self.bc[face], self.H[xi][0])
            for c in range(3):
                rv[c] += float(out["sat_v"][c])
            for c in range(6):
                e[c] += float(out["sat_e"][c])
        return apply_P(rv, e, J, mat)

    def rk_stage_at(self, node, stage, dt, fstate, fdq):
        """Fused low-storage stage at one node: (Q_out, dQ_out) from Q_in = fstate, dQ_in = fdq."""
        L = self.rhs_at(node, fstate)
        q = np.array([float(np.broadcast_to(c, ())) for c in fstate(*node)])
        dq = np.array([float(np.broadcast_to(c, ())) for c in fdq(*node)])
        dq_out = rk.A[stage] * dq + dt * L
        return q + rk.B[stage] * dq_out, dq_out
