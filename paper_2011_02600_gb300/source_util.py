"""Moment tensor of a double-couple point source (Section 7.1, Eq. momententor_pointsource).

M = M0 (n d^T + d n^T) with n the fault normal and d the slip direction, written in
(x = east, y = north, z = up) from the standard (north, east, down) expressions.
Returned in Voigt order (Mxx, Myy, Mzz, Mxy, Mxz, Myz) for sbp_set_source.
"""
import math


def moment_tensor_voigt(strike, dip, rake, M0):
    sd, cd = math.sin(dip), math.cos(dip)
    ss, cs = math.sin(strike), math.cos(strike)
    sr, cr = math.sin(rake), math.cos(rake)
    n_ned = (-sd * ss, sd * cs, -cd)
    d_ned = (cr * cs + cd * sr * ss, cr * ss - cd * sr * cs, -sr * sd)
    n = (n_ned[1], n_ned[0], -n_ned[2])
    d = (d_ned[1], d_ned[0], -d_ned[2])

    def m(i, j):
        return M0 * (n[i] * d[j] + d[i] * n[j])
    return (m(0, 0), m(1, 1), m(2, 2), m(0, 1), m(0, 2), m(1, 2))
