"""Semi-discrete velocity-stress elastic operator on a curvilinear mesh (oracle).

Test infrastructure only; see ``oracle/__init__.py``.

State Q = (vx, vy, vz, sxx, syy, szz, sxy, sxz, syz), arrays [9][s][r][q].
Axis xi = 0, 1, 2 is q, r, s; it is array axis 2, 1, 0.

The scheme (Section 4.2, Eq. gen_hyp_transformed_discrete, with the penalties
of Section 5, Eq. gen_hyp_transformed_discrete_SAT):

    P~^-1 dQ/dt = sum_xi D-_xi F_xi(Q) + sum_xi B_xi(D+_xi Q) + sum SAT_{xi,i},

with P~ = J^-1 P, P = diag(rho^-1 I, C) (Eq. S matrix), F_xi and B_xi of
Eq. split_form with basis e_xi = J grad(xi) (Section 2.2; the three flux rows
printed under Eq. transformedEQ repeat the first row, the rows used are those
of Eq. split_form).  D- acts on the flux and D+ on the velocity (Remark
after Eq. gen_hyp_transformed_discrete).

``rhs_raw`` returns the right-hand side above, split into the velocity rows
(3) and the stress rows (6, Voigt order, engineering shear); ``rhs`` applies
P~ to give dQ/dt.

Penalties:
* free surface (Eq. SAT_free_surface): velocity rows only,
  +H_xi^-1 J|grad xi| T at xi = 0 and -H_xi^-1 J|grad xi| T at xi = 1, with
  T = sigma n (Eq. velocity_traction_rotation), n = grad xi/|grad xi|
  (Eq. normal_vector);
* general boundary condition with parameter gamma (Eq. BC_General2) through
  hat variables (Appendix A, Eq. data_hat), penalties G (Eq. penalty_terms),
  rotation back to x, y, z (Eq. rotate_back_forth), the SAT vector that
  follows it and Eq. SAT_General.

Reading: on faces marked free the free-surface penalty is used, not the
general one with gamma = 1 (which adds a dissipative stress penalty).  Edge
and corner nodes receive the penalties of every face they lie on (the sum
over xi and i in Eq. gen_hyp_transformed_discrete_SAT).
"""
import numpy as np

from .metrics import apply_axis
from .operators import traditional_op, upwind_pair

ARRAY_AXIS = (2, 1, 0)   # xi = q, r, s -> array axis


class Scheme:
    """1D operators of one order on each axis of the reference cube [0, 1]^3.

    operator: "upwind" (the dual pair D-, D+ of Table 1 with their closures) or "traditional"
    (the central operator D of Table 2, used as both D- and D+: the scheme the paper compares
    the upwind one with).
    """

    def __init__(self, order, nodes, operator="upwind"):
        self.order = order
        self.operator = operator
        self.nodes = tuple(nodes)        # (nq, nr, ns)
        self.H, self.Dm, self.Dp = [], [], []
        for N in self.nodes:
            if operator == "upwind":
                H, Dm, Dp = upwind_pair(order, N)
            elif operator == "traditional":
                H, D = traditional_op(order, N)
                Dm = Dp = D
            else:
                raise ValueError(f"unknown operator family {operator!r}")
            self.H.append(H)
            self.Dm.append(Dm)
            self.Dp.append(Dp)

    def weights3(self):
        """Diagonal of H = H_q (x) H_r (x) H_s as an [s][r][q] array."""
        return self.H[2][:, None, None] * self.H[1][None, :, None] * self.H[0][None, None, :]

    def face_weights(self, xi):
        """H weights of the two other axes on a face normal to xi, shaped like the face slice."""
        if xi == 0:
            return self.H[2][:, None] * self.H[1][None, :]
        if xi == 1:
            return self.H[2][:, None] * self.H[0][None, :]
        return self.H[1][:, None] * self.H[0][None, :]


def flux(a_xi, sig):
    """F_xi velocity rows of Eq. split_form with e_xi = a_xi."""
    ax, ay, az = a_xi
    sxx, syy, szz, sxy, sxz, syz = sig
    return (ax * sxx + ay * sxy + az * sxz,
            ax * sxy + ay * syy + az * syz,
            ax * sxz + ay * syz + az * szz)


def strain_rows(a_xi, dv):
    """B_xi rows 4-9 of Eq. split_form applied to dv = D+_xi v (Voigt, engineering shear)."""
    ex, ey, ez = a_xi
    return [ex * dv[0], ey * dv[1], ez * dv[2],
            ey * dv[0] + ex * dv[1],
            ez * dv[0] + ex * dv[2],
            ez * dv[1] + ey * dv[2]]


def hat_variables(v_e, T_e, Z, gamma, side):
    """Appendix A, Eq. data_hat: boundary data (vhat, That) for one local component.

    At xi = 0 the outgoing characteristic q = (Z v + T)/2 is preserved, at xi = 1
    p = (Z v - T)/2 (Eq. BC_hat_1bc); the boundary condition of Eq. BC_General2
    holds exactly (Eq. BC_hat_2bc).
    """
    if side == 0:
        q_e = 0.5 * (Z * v_e + T_e)
        return (1 + gamma) / Z * q_e, (1 - gamma) * q_e
    p_e = 0.5 * (Z * v_e - T_e)
    return (1 + gamma) / Z * p_e, -(1 - gamma) * p_e


def traction(sig, n):
    """T = sigma n (Eq. velocity_traction_rotation)."""
    sxx, syy, szz, sxy, sxz, syz = sig
    nx, ny, nz = n
    return (sxx * nx + sxy * ny + sxz * nz,
            sxy * nx + syy * ny + syz * nz,
            sxz * nx + syz * ny + szz * nz)


def impedances(rho, lam, mu):
    """Z_n = rho c_p, Z_m = Z_l = rho c_s (Section 3)."""
    return np.sqrt(rho * (lam + 2 * mu)), np.sqrt(rho * mu)


def local_basis(n):
    """Rows of R = (n; m; l) (Eq. velocity_traction_rotation): m from m0 by
    Gram-Schmidt, l = n x m.  m0 is the coordinate axis least aligned with n."""
    nx, ny, nz = n
    an = np.stack([np.abs(nx), np.abs(ny), np.abs(nz)])
    k = np.argmin(an, axis=0)
    m0 = [np.where(k == 0, 1.0, 0.0), np.where(k == 1, 1.0, 0.0), np.where(k == 2, 1.0, 0.0)]
    nm0 = nx * m0[0] + ny * m0[1] + nz * m0[2]
    m = [m0[c] - nm0 * n[c] for c in range(3)]
    mn = np.sqrt(m[0] ** 2 + m[1] ** 2 + m[2] ** 2)
    m = [mc / mn for mc in m]
    l = [ny * m[2] - nz * m[1], nz * m[0] - nx * m[2], nx * m[1] - ny * m[0]]
    return [list(n), m, l]


def face_penalty(v, sig, a_xi, rho, lam, mu, side, bc, H0, vstar=None, Tstar=None):
    """Penalty of one face at a set of face nodes (arrays of any common shape).

    side 0 is xi = 0, side 1 is xi = 1; H0 is the first (= last) diagonal entry
    of H_xi.  bc is ("free",) or ("char", gamma).  vstar/Tstar are optional
    boundary data (exact v and T); the penalties then act on v - vstar,
    T - Tstar, which is the same as imposing the boundary condition with the
    data of (vstar, Tstar).

    Returns dict: sat_v (3), sat_e (6) (contributions to the rows of rhs_raw),
    vT = v.T, G2Z = sum_eta |G_eta|^2/Z_eta, hat = sum_eta vhat_eta That_eta,
    anorm = J |grad xi|.
    """
    anorm = np.sqrt(a_xi[0] ** 2 + a_xi[1] ** 2 + a_xi[2] ** 2)
    n = [c / anorm for c in a_xi]
    T = traction(sig, n)
    dv = [v[c] - (vstar[c] if vstar is not None else 0.0) for c in range(3)]
    dT = [T[c] - (Tstar[c] if Tstar is not None else 0.0) for c in range(3)]
    vT = v[0] * T[0] + v[1] * T[1] + v[2] * T[2]
    zero = 0 * anorm
    out = dict(vT=vT, anorm=anorm, G2Z=zero, hat=zero,
               sat_v=[zero, zero, zero], sat_e=[zero] * 6)
    if bc[0] == "free":
        sgn = 1.0 if side == 0 else -1.0
        out["sat_v"] = [sgn * anorm * dT[c] / H0 for c in range(3)]
        return out
    gamma = bc[1]
    Zp, Zs = impedances(rho, lam, mu)
    R = local_basis(n)
    Z = (Zp, Zs, Zs)
    G_eta, Gt_eta, G2Z, hat = [], [], zero, zero
    for e in range(3):
        v_e = R[e][0] * dv[0] + R[e][1] * dv[1] + R[e][2] * dv[2]
        T_e = R[e][0] * dT[0] + R[e][1] * dT[1] + R[e][2] * dT[2]
        vh, Th = hat_variables(v_e, T_e, Z[e], gamma, side)
        if side == 0:                                           # Eq. penalty_terms
            G = 0.5 * Z[e] * (v_e - vh) - 0.5 * (T_e - Th)
        else:
            G = 0.5 * Z[e] * (v_e - vh) + 0.5 * (T_e - Th)
        G_eta.append(G)
        Gt_eta.append(G / Z[e])
        G2Z = G2Z + G * G / Z[e]
        hat = hat + vh * Th
    # rotate back: G = R^T (G_n, G_m, G_l)
    Gx = [sum(R[e][c] * G_eta[e] for e in range(3)) for c in range(3)]
    Gtx = [sum(R[e][c] * Gt_eta[e] for e in range(3)) for c in range(3)]
    sgn = -1.0 if side == 0 else 1.0
    nx, ny, nz = n
    sat_sig = [sgn * nx * Gtx[0], sgn * ny * Gtx[1], sgn * nz * Gtx[2],
               sgn * (ny * Gtx[0] + nx * Gtx[1]),
               sgn * (nz * Gtx[0] + nx * Gtx[2]),
               sgn * (nz * Gtx[1] + ny * Gtx[2])]
    # Eq. SAT_General: SAT_{xi,i} = -H_xi^-1 e J|grad xi| SAT_i
    out["sat_v"] = [-anorm * Gx[c] / H0 for c in range(3)]
    out["sat_e"] = [-anorm * sat_sig[c] / H0 for c in range(6)]
    out["G2Z"] = G2Z
    out["hat"] = hat
    return out


def face_slice(xi, side, N):
    idx = [slice(None)] * 3
    idx[ARRAY_AXIS[xi]] = 0 if side == 0 else N - 1
    return tuple(idx)


def rhs_raw(Q, scheme, a, mat, bc, data=None, with_sat=True, diag=None):
    """P~^-1 dQ/dt: (velocity rows [3], stress rows [6]).

    a: a[xi][eta] = J xi_eta; mat: (rho, lam, mu) arrays; bc: six face
    conditions (q0, q1, r0, r1, s0, s1); data: optional function
    face -> (vstar, Tstar) of boundary data; diag: optional dict filled with
    per-face diagnostics.
    """
    v = Q[0:3]
    sig = Q[3:9]
    rv = [np.zeros_like(v[0]) for _ in range(3)]
    e = [np.zeros_like(v[0]) for _ in range(6)]
    for xi in range(3):
        ax = ARRAY_AXIS[xi]
        F = flux(a[xi], sig)                                  # conservative flux
        for c in range(3):
            rv[c] += apply_axis(scheme.Dm[xi], F[c], ax)      # D- on the flux
        dv = [apply_axis(scheme.Dp[xi], v[c], ax) for c in range(3)]   # D+ on v
        B = strain_rows(a[xi], dv)                            # B_xi rows
        for c in range(6):
            e[c] += B[c]
    if with_sat:
        for face in range(6):
            if bc[face][0] == "interface":      # coupled to another block: multiblock.py adds it
                continue
            xi, side = divmod(face, 2)
            sl = face_slice(xi, side, scheme.nodes[xi])
            vs, Ts = (None, None)
            if data is not None:
                vs, Ts = data(face)
            out = face_penalty([c[sl] for c in v], [c[sl] for c in sig],
                               [c[sl] for c in a[xi]], *[m[sl] for m in mat],
                               side, bc[face], scheme.H[xi][0], vs, Ts)
            for c in range(3):
                rv[c][sl] += out["sat_v"][c]
            for c in range(6):
                e[c][sl] += out["sat_e"][c]
            if diag is not None:
                diag[face] = out
    return rv, e


def apply_P(rv, e, J, mat):
    """dQ/dt = P~ (P~^-1 dQ/dt): velocity rows / (rho J), stress rows C e / J."""
    rho, lam, mu = mat
    dv = [rv[c] / (rho * J) for c in range(3)]
    tr = e[0] + e[1] + e[2]
    ds = [(lam * tr + 2 * mu * e[0]) / J, (lam * tr + 2 * mu * e[1]) / J, (lam * tr + 2 * mu * e[2]) / J,
          mu * e[3] / J, mu * e[4] / J, mu * e[5] / J]
    return np.stack(dv + ds)


def rhs(Q, scheme, J, a, mat, bc, data=None):
    """dQ/dt of the semi-discrete scheme with penalties."""
    rv, e = rhs_raw(Q, scheme, a, mat, bc, data)
    return apply_P(rv, e, J, mat)


def energy(Q, scheme, J, mat):
    """Discrete energy (Eq. physical_energy_discrete) with P~ in place of P:
    E = 1/2 <Q, P~^-1 Q>_H = 1/2 sum H J (rho |v|^2 + sigma^T S sigma).

    S = C^-1: sigma^T S sigma = [sum s_ii^2 + 2 sum s_ij^2 - lam/(3 lam + 2 mu) tr^2] / (2 mu).
    """
    rho, lam, mu = mat
    v = Q[0:3]
    s = Q[3:9]
    tr = s[0] + s[1] + s[2]
    sSs = (s[0] ** 2 + s[1] ** 2 + s[2] ** 2 + 2 * (s[3] ** 2 + s[4] ** 2 + s[5] ** 2)
           - lam / (3 * lam + 2 * mu) * tr ** 2) / (2 * mu)
    dens = J * (rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) + sSs)
    return 0.5 * float(np.sum(scheme.weights3() * dens))


def inner_H(Q, rv, e, scheme):
    """<Q, (rv, e)>_H with the Voigt pairing of the stress rows."""
    W = scheme.weights3()
    tot = sum(Q[c] * rv[c] for c in range(3)) + sum(Q[3 + c] * e[c] for c in range(6))
    return float(np.sum(W * tot))


def surface_integral(values, scheme, xi, anorm):
    """I_{xi_i}(f) of Eq. surface_cubature_1D on one face: sum J|grad xi| f h h."""
    return float(np.sum(scheme.face_weights(xi) * anorm * values))
