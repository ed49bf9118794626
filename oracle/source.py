"""Moment-tensor point source (oracle).

Test infrastructure only; see ``oracle/__init__.py``.

Section 7.1, Eq. momententor_pointsource: f = M delta(x - x_p) g(t).  The
paper discretises the singular source "to high order" after Petersson et al.
(2016) without describing it.  Reading taken here:

* The stress equation receives -M g(t) delta_h (moment-rate convention:
  g integrates to one for the LOH1 time function).
* delta_h at node (i, j, k) = phi_i phi_j phi_k / (J_ijk H_q,i H_r,j H_s,k),
  so that sum H J delta_h f = sum phi phi phi f.  Each 1D weight vector phi
  lives on m+1 consecutive nodes starting at floor(xi_0/h) - (m-1)/2 (centred
  on the cell holding the source, shifted inwards at a face) and satisfies
  the discrete moment conditions
  sum_i phi_i (xi_i - xi_0)^k = delta_k0 for k = 0..m, with m = order + 1.
* The moment tensor of a double couple is M = M0 (n d^T + d n^T) with n the
  fault normal and d the slip direction.
"""
import math

import numpy as np


def delta_weights_1d(xi0, N, m):
    """(first node index, phi[0..m]) of the 1D discrete delta at reference coordinate xi0."""
    h = 1.0 / (N - 1)
    c = int(np.floor(xi0 / h)) - (m - 1) // 2     # m + 1 nodes centred on the source's cell
    c = max(0, min(N - 1 - m, c))
    xs = (np.arange(c, c + m + 1) * h - xi0) / h
    V = np.vander(xs, m + 1, increasing=True).T      # V[k, i] = xs_i^k
    rhs = np.zeros(m + 1)
    rhs[0] = 1.0
    return c, np.linalg.solve(V, rhs)


def slip_and_normal(strike, dip, rake):
    """Fault normal n and slip direction d in (x=east, y=north, z=up), angles in radians.

    From the standard (north, east, down) expressions of Aki & Richards:
    n = (-sin(dip) sin(strike), sin(dip) cos(strike), -cos(dip)),
    d = (cos(rake) cos(strike) + cos(dip) sin(rake) sin(strike),
         cos(rake) sin(strike) - cos(dip) sin(rake) cos(strike),
         -sin(rake) sin(dip)).
    """
    sd, cd = math.sin(dip), math.cos(dip)
    ss, cs = math.sin(strike), math.cos(strike)
    sr, cr = math.sin(rake), math.cos(rake)
    n_ned = np.array([-sd * ss, sd * cs, -cd])
    d_ned = np.array([cr * cs + cd * sr * ss, cr * ss - cd * sr * cs, -sr * sd])

    def to_enu(v):
        return np.array([v[1], v[0], -v[2]])
    return to_enu(n_ned), to_enu(d_ned)


def moment_tensor(strike, dip, rake, M0):
    """Voigt (Mxx, Myy, Mzz, Mxy, Mxz, Myz) of M = M0 (n d^T + d n^T)."""
    n, d = slip_and_normal(strike, dip, rake)
    M = M0 * (np.outer(n, d) + np.outer(d, n))
    return np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])


def ricker(t, f0, t0):
    """(1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0."""
    a = (math.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def loh1_stf(t, T=0.1):
    """g(t) = t/T^2 exp(-t/T) (Eq. momententor_pointsource)."""
    return t / T ** 2 * math.exp(-t / T) if t > 0 else 0.0


class PointSource:
    """Discrete point source: node box, weights, moment tensor and time function."""

    def __init__(self, ref_xyz, Mv, stf, order, nodes, Hdiag, J):
        self.Mv = np.asarray(Mv, dtype=float)
        self.stf = stf
        m = order + 1
        self.box = []
        phis = []
        for ax in range(3):
            c, phi = delta_weights_1d(ref_xyz[ax], nodes[ax], m)
            self.box.append(c)
            phis.append(phi)
        i0, j0, k0 = self.box
        sl = (slice(k0, k0 + m + 1), slice(j0, j0 + m + 1), slice(i0, i0 + m + 1))
        self.sl = sl
        w = phis[2][:, None, None] * phis[1][None, :, None] * phis[0][None, None, :]
        self.delta = w / (J[sl] * Hdiag[sl])

    def add_to(self, dQdt, t):
        """dQ/dt[stress] += -M g(t) delta_h."""
        g = self.stf(t)
        for c in range(6):
            dQdt[3 + c][self.sl] -= self.Mv[c] * g * self.delta
        return dQdt
