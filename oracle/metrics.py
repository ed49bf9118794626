"""Jacobian and metric terms of the curvilinear map (oracle).

Test infrastructure only; see ``oracle/__init__.py``.

Section 2.2: J = x_q (y_r z_s - z_r y_s) - y_q (x_r z_s - z_r x_s)
+ z_q (x_r y_s - y_r x_s), and the metric derivatives xi_eta by Cramer's rule.
The printed q_z is garbled; the cofactor is (x_r y_s - y_r x_s)/J, which is
what is used.  The basis vectors of Eq. split_form are e_xi = J (xi_x, xi_y,
xi_z) (the equation after eq. conservative), so a[xi][eta] = J xi_eta.

Reading (the paper is silent): the derivatives x_q ... z_s are taken with
D_c = (D+ + D-)/2 of the same order along each reference axis.
"""
import numpy as np
import scipy.sparse as sp

from .operators import upwind_pair


def apply_axis(D, f, axis):
    """Apply the 1D operator D (dense or sparse, N x N) along ``axis`` of array f."""
    Ds = sp.csr_matrix(D)
    g = np.moveaxis(f, axis, 0)
    shp = g.shape
    out = Ds @ g.reshape(shp[0], -1)
    return np.moveaxis(np.asarray(out).reshape(shp), 0, axis)


def central_ops(order, nodes):
    """D_c = (D+ + D-)/2 on each axis of the unit reference cube (spacing 1/(N-1))."""
    ops = []
    for N in nodes:
        _, Dm, Dp = upwind_pair(order, N)
        ops.append(0.5 * (Dp + Dm))
    return ops


def metrics(x, y, z, order):
    """J and a[xi][eta] = J xi_eta for coordinate arrays x, y, z laid out [s][r][q].

    Returns (J, a) with a a 3x3 nested list indexed a[xi][eta], xi in (q, r, s),
    eta in (x, y, z).
    """
    nodes = (x.shape[2], x.shape[1], x.shape[0])
    Dq, Dr, Ds = central_ops(order, nodes)

    def d(f):
        return apply_axis(Dq, f, 2), apply_axis(Dr, f, 1), apply_axis(Ds, f, 0)

    x_q, x_r, x_s = d(x)
    y_q, y_r, y_s = d(y)
    z_q, z_r, z_s = d(z)
    return jacobian_and_metrics(x_q, x_r, x_s, y_q, y_r, y_s, z_q, z_r, z_s)


def jacobian_and_metrics(x_q, x_r, x_s, y_q, y_r, y_s, z_q, z_r, z_s):
    """J and a[xi][eta] = J xi_eta from the nine coordinate derivatives (Section 2.2)."""
    J = x_q * (y_r * z_s - z_r * y_s) - y_q * (x_r * z_s - z_r * x_s) + z_q * (x_r * y_s - y_r * x_s)
    q_x = (y_r * z_s - z_r * y_s) / J
    q_y = (z_r * x_s - x_r * z_s) / J
    q_z = (x_r * y_s - y_r * x_s) / J
    r_x = (z_q * y_s - y_q * z_s) / J
    r_y = (x_q * z_s - z_q * x_s) / J
    r_z = (y_q * x_s - y_s * x_q) / J
    s_x = (y_q * z_r - z_q * y_r) / J
    s_y = (z_q * x_r - x_q * z_r) / J
    s_z = (x_q * y_r - x_r * y_q) / J
    a = [[J * q_x, J * q_y, J * q_z],
         [J * r_x, J * r_y, J * r_z],
         [J * s_x, J * s_y, J * s_z]]
    return J, a
