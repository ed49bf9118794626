"""Two curvilinear blocks coupled at a shared face by interface penalties (oracle).

Test infrastructure only; see ``oracle/__init__.py``.

Section 7.1 splits the LOH1 domain into two blocks at the material discontinuity and couples
the blocks weakly with penalties; the paper writes the penalty construction out for physical
boundaries (Appendix A, Eq. penalty_terms, Eq. data_hat) and says that the hat variables solve a
Riemann problem constrained by the physical conditions.  Reading (the interface version is not
printed): at a locked interface the conditions are continuity of particle velocity and of
traction, v- = v+ and T- = T+, with T = sigma n for the one unit normal n of the shared face.
Block "-" has the shared face at xi = 1 (its outgoing characteristic there is Z v - T), block
"+" has it at xi = 0 (outgoing: Z v + T).  Per local component (n, m, l) with impedances
Z = (Z_p, Z_s, Z_s) of each side, the hat variables keep both outgoing characteristics and
satisfy the interface conditions:
    Z- vhat - That = Z- v- - T-,     Z+ vhat + That = Z+ v+ + T+.
Each block then receives the penalty of Eq. penalty_terms / Eq. SAT_General with these hat
variables in place of the boundary's, on its own face.
"""
import numpy as np

from .elastic import (ARRAY_AXIS, apply_P, face_slice, impedances, inner_H, local_basis, rhs_raw,
                      surface_integral, traction)


def interface_hat(v_m, T_m, Z_m, v_p, T_p, Z_p):
    """Hat values (vhat, That) of one local component at a locked interface: block "-" at its
    xi = 1 face (v_m, T_m, Z_m), block "+" at its xi = 0 face (v_p, T_p, Z_p)."""
    vh = (Z_m * v_m - T_m + Z_p * v_p + T_p) / (Z_m + Z_p)
    Th = Z_m * vh - (Z_m * v_m - T_m)
    return vh, Th


def interface_penalty(v, sig, a_xi, mat, side, H0, v_o, sig_o, mat_o):
    """Penalty of one block's interface face (arrays over the face nodes).  side 1: this block is
    "-" (its face at xi = 1); side 0: this block is "+".  v_o, sig_o, mat_o: the other block's
    velocity, stress and (rho, lam, mu) at the same face nodes.  The unit normal n = a/|a| is
    this block's (the other block's is the same: both follow from the shared face's nodes).
    Returns the same dict as elastic.face_penalty (sat_v, sat_e, G2Z, hat, anorm)."""
    anorm = np.sqrt(a_xi[0] ** 2 + a_xi[1] ** 2 + a_xi[2] ** 2)
    n = [c / anorm for c in a_xi]
    T, T_o = traction(sig, n), traction(sig_o, n)
    Zp, Zs = impedances(*mat)
    Zp_o, Zs_o = impedances(*mat_o)
    R = local_basis(n)
    Z, Z_o = (Zp, Zs, Zs), (Zp_o, Zs_o, Zs_o)
    zero = 0 * anorm
    G_eta, Gt_eta, G2Z, hat = [], [], zero, zero
    for e in range(3):
        v_e = R[e][0] * v[0] + R[e][1] * v[1] + R[e][2] * v[2]
        T_e = R[e][0] * T[0] + R[e][1] * T[1] + R[e][2] * T[2]
        vo_e = R[e][0] * v_o[0] + R[e][1] * v_o[1] + R[e][2] * v_o[2]
        To_e = R[e][0] * T_o[0] + R[e][1] * T_o[1] + R[e][2] * T_o[2]
        if side == 1:
            vh, Th = interface_hat(v_e, T_e, Z[e], vo_e, To_e, Z_o[e])
            G = 0.5 * Z[e] * (v_e - vh) + 0.5 * (T_e - Th)       # Eq. penalty_terms, xi = 1
        else:
            vh, Th = interface_hat(vo_e, To_e, Z_o[e], v_e, T_e, Z[e])
            G = 0.5 * Z[e] * (v_e - vh) - 0.5 * (T_e - Th)       # Eq. penalty_terms, xi = 0
        G_eta.append(G)
        Gt_eta.append(G / Z[e])
        G2Z = G2Z + G * G / Z[e]
        hat = hat + vh * Th
    Gx = [sum(R[e][c] * G_eta[e] for e in range(3)) for c in range(3)]
    Gtx = [sum(R[e][c] * Gt_eta[e] for e in range(3)) for c in range(3)]
    sgn = -1.0 if side == 0 else 1.0
    nx, ny, nz = n
    sat_sig = [sgn * nx * Gtx[0], sgn * ny * Gtx[1], sgn * nz * Gtx[2],
               sgn * (ny * Gtx[0] + nx * Gtx[1]),
               sgn * (nz * Gtx[0] + nx * Gtx[2]),
               sgn * (nz * Gtx[1] + ny * Gtx[2])]
    return dict(sat_v=[-anorm * Gx[c] / H0 for c in range(3)], sat_e=[-anorm * sat_sig[c] / H0 for c in range(6)],
                G2Z=G2Z, hat=hat, anorm=anorm)


def two_block_rhs_raw(Qm, Qp, sch_m, sch_p, a_m, a_p, mat_m, mat_p, bc_m, bc_p, xi, diag=None):
    """P~^-1 dQ/dt of both blocks: block "-" (Qm) has the shared face at xi = 1, block "+" (Qp)
    at xi = 0 (bc_m[2 xi + 1] and bc_p[2 xi] are ("interface",)).  The shared faces must hold the
    same nodes in the same order.  diag (optional dict) receives the two faces' penalty dicts
    under "-" and "+"."""
    assert bc_m[2 * xi + 1][0] == "interface" and bc_p[2 * xi][0] == "interface"
    rv_m, e_m = rhs_raw(Qm, sch_m, a_m, mat_m, bc_m)
    rv_p, e_p = rhs_raw(Qp, sch_p, a_p, mat_p, bc_p)
    sl_m = face_slice(xi, 1, sch_m.nodes[xi])
    sl_p = face_slice(xi, 0, sch_p.nodes[xi])
    fm = [c[sl_m] for c in Qm]
    fp = [c[sl_p] for c in Qp]
    mm = [m[sl_m] for m in mat_m]
    mp = [m[sl_p] for m in mat_p]
    out_m = interface_penalty(fm[0:3], fm[3:9], [c[sl_m] for c in a_m[xi]], mm, 1, sch_m.H[xi][0],
                              fp[0:3], fp[3:9], mp)
    out_p = interface_penalty(fp[0:3], fp[3:9], [c[sl_p] for c in a_p[xi]], mp, 0, sch_p.H[xi][0],
                              fm[0:3], fm[3:9], mm)
    for rv, e, out, sl in ((rv_m, e_m, out_m, sl_m), (rv_p, e_p, out_p, sl_p)):
        for c in range(3):
            rv[c][sl] += out["sat_v"][c]
        for c in range(6):
            e[c][sl] += out["sat_e"][c]
    if diag is not None:
        diag["-"], diag["+"] = out_m, out_p
    return (rv_m, e_m), (rv_p, e_p)


def two_block_rhs(Qm, Qp, sch_m, sch_p, J_m, J_p, a_m, a_p, mat_m, mat_p, bc_m, bc_p, xi):
    """dQ/dt of both blocks (Eq. gen_hyp_transformed_discrete_SAT with the interface penalties)."""
    (rm, em), (rp, ep) = two_block_rhs_raw(Qm, Qp, sch_m, sch_p, a_m, a_p, mat_m, mat_p, bc_m, bc_p, xi)
    return apply_P(rm, em, J_m, mat_m), apply_P(rp, ep, J_p, mat_p)


def interface_energy_rate(Qm, Qp, sch_m, sch_p, a_m, a_p, mat_m, mat_p, bc_m, bc_p, xi):
    """(<Qm, P~^-1 dQm/dt>_H + <Qp, P~^-1 dQp/dt>_H, its prediction from the interface alone:
    -I(sum |G|^2/Z) on both faces plus I(vhat That) on the "-" face minus the same on the "+"
    face), for blocks whose other faces are free surfaces (which contribute nothing)."""
    diag = {}
    (rm, em), (rp, ep) = two_block_rhs_raw(Qm, Qp, sch_m, sch_p, a_m, a_p, mat_m, mat_p, bc_m, bc_p, xi, diag)
    lhs = inner_H(Qm, rm, em, sch_m) + inner_H(Qp, rp, ep, sch_p)
    dm, dp = diag["-"], diag["+"]
    want = (-surface_integral(dm["G2Z"], sch_m, xi, dm["anorm"]) - surface_integral(dp["G2Z"], sch_p, xi, dp["anorm"])
            + surface_integral(dm["hat"], sch_m, xi, dm["anorm"]) - surface_integral(dp["hat"], sch_p, xi, dp["anorm"]))
    return lhs, want, diag


def array_axis(xi):
    return ARRAY_AXIS[xi]
