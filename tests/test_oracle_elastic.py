"""Pins of the oracle's semi-discrete scheme against the paper's lemmas and
theorems (Sections 2, 4, 5, 6, Appendix A) and against closed forms."""
import math

import numpy as np
import pytest

from oracle import rk
from oracle.elastic import (Scheme, apply_P, energy, face_penalty, flux, hat_variables,
                            inner_H, rhs, rhs_raw, strain_rows, surface_integral)
from oracle.metrics import metrics
from oracle.operators import CLOSURE, TABLE1, TRADITIONAL
from oracle.pointwise import PointOracle
from workloads.fields import gaussian_pulse, random_state, smooth_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium


def _grid(order, nodes=None, geometry="curvy", ext=(1.0, 1.2, 0.9)):
    if nodes is None:   # orders 8, 9 need 21 nodes per axis (two 8-row closures + reach 5)
        nodes = (16, 17, 18) if order <= 7 else (21, 22, 23)
    x, y, z = node_coordinates(make_map(geometry, ext), nodes)
    J, a = metrics(x, y, z, order)
    return x, y, z, J, a


def _random_medium(shape, seed=3):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(1.0, 2.0, shape)
    mu = rng.uniform(0.5, 1.5, shape)
    lam = rng.uniform(0.2, 2.0, shape)
    return rho, lam, mu


def _faces_sum(diag, key, scheme, signed):
    tot = 0.0
    for f in range(6):
        s = (1.0 if f % 2 else -1.0) if signed else 1.0
        tot += s * surface_integral(diag[f][key], scheme, f // 2, diag[f]["anorm"])
    return tot


def test_antisymmetry_lemma_pointwise():
    """Lemma (anti-symmetric form): (dQ)^T F_xi(Q) - Q^T B_xi(dQ) = 0 for any basis vector."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.normal(size=3)
        Q = rng.normal(size=9)
        dQ = rng.normal(size=9)
        F = flux(a, Q[3:9])
        B = strain_rows(a, dQ[0:3])
        val = sum(dQ[c] * F[c] for c in range(3)) - sum(Q[3 + c] * B[c] for c in range(6))
        assert abs(val) < 1e-13


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7, 8, 9])
def test_semidiscrete_energy_without_penalties(order):
    """Theorem (semi-discrete energy): <Q, P~^-1 dQ/dt>_H = I(v^T T) before penalties."""
    x, y, z, J, a = _grid(order)
    sch = Scheme(order, J.shape[::-1])
    mat = _random_medium(J.shape)
    Q = random_state(sch.nodes, 11, 1.0, 1.0)
    diag = {}
    rhs_raw(Q, sch, a, mat, [("free",)] * 6, diag=diag)
    rv, e = rhs_raw(Q, sch, a, mat, [("free",)] * 6, with_sat=False)
    lhs = inner_H(Q, rv, e, sch)
    want = _faces_sum(diag, "vT", sch, signed=True)
    assert abs(lhs - want) < 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7, 8, 9])
def test_free_surface_scheme_conserves_energy(order):
    """Theorem (free-surface procedure): d/dt ||Q||^2_HP = 0, i.e. <Q, P~^-1 dQ/dt>_H = 0
    for random Q, random medium, every face free, fully curvilinear mesh."""
    x, y, z, J, a = _grid(order)
    sch = Scheme(order, J.shape[::-1])
    mat = _random_medium(J.shape)
    Q = random_state(sch.nodes, 12, 1.0, 1.0)
    rv, e = rhs_raw(Q, sch, a, mat, [("free",)] * 6)
    W = sch.weights3()
    scale = sum(np.sum(np.abs(W * Q[c] * rv[c])) for c in range(3))
    assert abs(inner_H(Q, rv, e, sch)) < 1e-14 * scale


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7, 8, 9])
def test_general_bc_energy_identity(order):
    """Theorem (general boundary conditions): <Q, P~^-1 dQ/dt>_H = F_luc + I(vhat^T That),
    with F_luc and the hat term evaluated separately, gamma in [-1, 1] per face."""
    x, y, z, J, a = _grid(order)
    sch = Scheme(order, J.shape[::-1])
    mat = _random_medium(J.shape)
    Q = random_state(sch.nodes, 13, 1.0, 1.0)
    bc = [("char", g) for g in (0.0, 0.4, -0.6, 1.0, -1.0, 0.25)]
    diag = {}
    rv, e = rhs_raw(Q, sch, a, mat, bc, diag=diag)
    lhs = inner_H(Q, rv, e, sch)
    Fluc = -_faces_sum(diag, "G2Z", sch, signed=False)
    Ihat = _faces_sum(diag, "hat", sch, signed=True)
    assert Fluc <= 0 and Ihat <= 1e-12
    assert abs(lhs - (Fluc + Ihat)) < 1e-12 * abs(Fluc)


@pytest.mark.parametrize("order", [4, 6])
def test_workload_boundary_mix_dissipates(order):
    """Top face free, the others absorbing (gamma = 0): <Q, P~^-1 dQ/dt>_H equals the
    absorbing faces' F_luc + hat terms and is never positive."""
    x, y, z, J, a = _grid(order)
    sch = Scheme(order, J.shape[::-1])
    mat = _random_medium(J.shape)
    Q = random_state(sch.nodes, 14, 1.0, 1.0)
    bc = [("char", 0.0)] * 5 + [("free",)]
    diag = {}
    rv, e = rhs_raw(Q, sch, a, mat, bc, diag=diag)
    lhs = inner_H(Q, rv, e, sch)
    want = 0.0
    for f in range(5):
        s = 1.0 if f % 2 else -1.0
        want += -surface_integral(diag[f]["G2Z"], sch, f // 2, diag[f]["anorm"])
        want += s * surface_integral(diag[f]["hat"], sch, f // 2, diag[f]["anorm"])
    assert lhs <= 0 and abs(lhs - want) < 1e-12 * abs(want)


def test_hat_variables_closed_form():
    """Appendix A: hat data satisfy the boundary condition exactly, keep the outgoing
    characteristic, and vhat That = +-(1 - gamma^2)/Z * (outgoing)^2."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        v, T = rng.normal(size=2)
        Z = rng.uniform(0.5, 3.0)
        g = rng.uniform(-1, 1)
        vh, Th = hat_variables(v, T, Z, g, 0)
        assert abs(0.5 * Z * (1 - g) * vh - 0.5 * (1 + g) * Th) < 1e-13
        assert abs(0.5 * (Z * vh + Th) - 0.5 * (Z * v + T)) < 1e-13
        qv = 0.5 * (Z * v + T)
        assert abs(vh * Th - (1 - g * g) / Z * qv * qv) < 1e-12 and vh * Th >= -1e-15
        vh, Th = hat_variables(v, T, Z, g, 1)
        assert abs(0.5 * Z * (1 - g) * vh + 0.5 * (1 + g) * Th) < 1e-13
        assert abs(0.5 * (Z * vh - Th) - 0.5 * (Z * v - T)) < 1e-13
        pv = 0.5 * (Z * v - T)
        assert abs(vh * Th + (1 - g * g) / Z * pv * pv) < 1e-12 and vh * Th <= 1e-15


def test_absorbing_penalty_is_incoming_characteristic():
    """gamma = 0: G reduces to the incoming characteristic (p at xi = 0, q at xi = 1);
    a state whose incoming characteristic vanishes receives no penalty."""
    rng = np.random.default_rng(6)
    n = rng.normal(size=3)
    a_xi = list(n * 2.0)
    rho, lam, mu = 2.0, 1.5, 1.0
    Zp, Zs = math.sqrt(rho * (lam + 2 * mu)), math.sqrt(rho * mu)
    nn = n / np.linalg.norm(n)
    # a P-wave leaving through xi = 0 (moving against n): v = -c n, sigma = (lam I + 2 mu n n^T) c' ...
    # choose sigma with T = Z_p v_n n (so p_n = (Z v - T)/2 = 0) and no tangential part
    vn = 0.7
    v = list(vn * nn)
    T = Zp * vn * nn
    Smat = np.outer(T, nn) + np.outer(nn, T) - np.dot(T, nn) * np.outer(nn, nn)
    sig = [Smat[0, 0], Smat[1, 1], Smat[2, 2], Smat[0, 1], Smat[0, 2], Smat[1, 2]]
    out = face_penalty(v, sig, a_xi, rho, lam, mu, 0, ("char", 0.0), 1.0)
    assert max(abs(x) for x in out["sat_v"] + out["sat_e"]) < 1e-12
    out1 = face_penalty(v, sig, a_xi, rho, lam, mu, 1, ("char", 0.0), 1.0)
    assert max(abs(x) for x in out1["sat_v"]) > 0.1


def _poly_fields(X, rng, quadratic):
    """Random polynomial fields of degree <= 2 in x and their gradients."""
    vals, grads = [], []
    for _ in range(9):
        b = rng.normal()
        g = rng.normal(size=3)
        K = rng.normal(size=(3, 3)) if quadratic else np.zeros((3, 3))
        K = 0.5 * (K + K.T)
        f = b + sum(g[i] * X[i] for i in range(3)) + 0.5 * sum(K[i, j] * X[i] * X[j] for i in range(3) for j in range(3))
        gr = [g[i] + sum(K[i, j] * X[j] for j in range(3)) for i in range(3)]
        vals.append(f)
        grads.append(gr)
    return vals, grads


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_polynomial_state_reproduces_continuous_equations(order):
    """On an affine mesh, fields of degree <= p are differentiated exactly by D+- at every node, so
    dQ/dt (penalties off) must equal the textbook velocity-stress equations (Eq. elastic_sys):
    rho dv_i/dt = d sigma_ij/dx_j, d sigma/dt = lam tr(grad v) I + mu (grad v + grad v^T)."""
    nodes = (16, 17, 18)
    rng = np.random.default_rng(order)
    A = np.eye(3) + rng.normal(scale=0.15, size=(3, 3))
    nq, nr, ns = nodes
    qq = (np.arange(nq) / (nq - 1))[None, None, :]
    rr = (np.arange(nr) / (nr - 1))[None, :, None]
    ss = (np.arange(ns) / (ns - 1))[:, None, None]
    shape = (ns, nr, nq)
    X = [np.broadcast_to(A[i, 0] * qq + A[i, 1] * rr + A[i, 2] * ss + 0.3 * i, shape).copy() for i in range(3)]
    J, a = metrics(*X, order)
    sch = Scheme(order, nodes)
    mat = _random_medium(shape, seed=order)
    vals, grads = _poly_fields(X, rng, quadratic=order >= 4)
    Q = np.stack(vals)
    rv, e = rhs_raw(Q, sch, a, mat, [("free",)] * 6, with_sat=False)
    got = apply_P(rv, e, J, mat)
    rho, lam, mu = mat
    idx = {(0, 0): 3, (1, 1): 4, (2, 2): 5, (0, 1): 6, (1, 0): 6, (0, 2): 7, (2, 0): 7, (1, 2): 8, (2, 1): 8}
    gv = [[grads[i][j] for j in range(3)] for i in range(3)]      # dv_i/dx_j
    div = [sum(grads[idx[(i, j)]][j] for j in range(3)) for i in range(3)]
    tr = gv[0][0] + gv[1][1] + gv[2][2]
    want = [div[i] / rho for i in range(3)]
    want += [lam * tr + 2 * mu * gv[i][i] for i in range(3)]
    want += [mu * (gv[0][1] + gv[1][0]), mu * (gv[0][2] + gv[2][0]), mu * (gv[1][2] + gv[2][1])]
    for c in range(9):
        scale = np.abs(want[c]).max()
        assert np.abs(got[c] - want[c]).max() < 1e-9 * scale, c


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7, 8, 9])
def test_linearity(order):
    x, y, z, J, a = _grid(order)
    sch = Scheme(order, J.shape[::-1])
    mat = _random_medium(J.shape)
    bc = [("char", 0.0)] * 5 + [("free",)]
    Q1 = random_state(sch.nodes, 1)
    Q2 = random_state(sch.nodes, 2)
    r12 = rhs(2.0 * Q1 - 3.0 * Q2, sch, J, a, mat, bc)
    r = 2.0 * rhs(Q1, sch, J, a, mat, bc) - 3.0 * rhs(Q2, sch, J, a, mat, bc)
    assert np.abs(r12 - r).max() < 1e-12 * np.abs(r).max()


def _run_energy(order, nodes, dt, T, bc):
    x, y, z = node_coordinates(make_map("curvy", (1.0, 1.0, 1.0), eps=0.05), nodes)
    J, a = metrics(x, y, z, order)
    sch = Scheme(order, nodes)
    mat = (np.full(J.shape, 1.0), np.full(J.shape, 1.0), np.full(J.shape, 1.0))
    Q = np.stack(gaussian_pulse(x, y, z, (0.5, 0.5, 0.5), 0.15))
    dQ = np.zeros_like(Q)
    E0 = energy(Q, sch, J, mat)
    n = int(round(T / dt))
    Es = [E0]
    for k in range(n):
        rk.rk_step(Q, dQ, k * dt, dt, lambda q, t: rhs(q, sch, J, a, mat, bc))
        Es.append(energy(Q, sch, J, mat))
    return np.array(Es)


def test_fully_discrete_energy_drift_fifth_order():
    """All faces free: the semi-discrete energy is constant, so the fully discrete drift
    comes from RK4 only and falls like dt^5 (|R(iy)|^2 = 1 - 7 y^6/1800 + ...)."""
    nodes = (13, 13, 13)
    d1 = _run_energy(4, nodes, 0.02, 0.2, [("free",)] * 6)
    d2 = _run_energy(4, nodes, 0.01, 0.2, [("free",)] * 6)
    e1 = abs(d1[-1] - d1[0]) / d1[0]
    e2 = abs(d2[-1] - d2[0]) / d2[0]
    assert d1[-1] <= d1[0] and e1 < 1e-4
    assert 28 < e1 / e2 < 36, (e1, e2)


def test_absorbing_energy_non_increasing():
    Es = _run_energy(6, (17, 17, 17), 0.01, 0.3, [("char", 0.0)] * 5 + [("free",)])
    assert np.all(np.diff(Es) <= 1e-14 * Es[0])
    assert Es[-1] < Es[0]


def _plane_wave(kind, X, t, rho, lam, mu, dvec, pol, wl):
    """Exact plane wave of Section 6.2's kind in 3D: P (pol = d) or S (pol _|_ d),
    u = pol F(d.x - c t), F = sin(2 pi phi / wl); returns v, sigma (Voigt)."""
    c = math.sqrt((lam + 2 * mu) / rho) if kind == "P" else math.sqrt(mu / rho)
    phi = dvec[0] * X[0] + dvec[1] * X[1] + dvec[2] * X[2] - c * t
    k = 2 * math.pi / wl
    Fp = k * np.cos(k * phi)                       # F'(phi)
    v = [-c * pol[i] * Fp for i in range(3)]
    E = 0.5 * (np.outer(pol, dvec) + np.outer(dvec, pol))
    tr = np.trace(E)
    S = lam * tr * np.eye(3) + 2 * mu * E
    sig = [S[0, 0] * Fp, S[1, 1] * Fp, S[2, 2] * Fp, S[0, 1] * Fp, S[0, 2] * Fp, S[1, 2] * Fp]
    return v, sig


def _mms_error(order, n, kind, T=0.25, bc=None, wl=1.6, operator="upwind"):
    nodes = (n + 1, n + 1, n + 1)
    fmap = make_map("curvy", (1.0, 1.0, 1.0), eps=0.05)
    X = node_coordinates(fmap, nodes)
    J, a = metrics(*X, order)
    sch = Scheme(order, nodes, operator)
    rho, lam, mu = 1.0, 2.0, 1.0
    mat = tuple(np.full(J.shape, v) for v in (rho, lam, mu))
    dvec = np.array([1.0, 2.0, 2.0]) / 3.0
    pol = dvec if kind == "P" else np.array([2.0, -1.0, 0.0]) / math.sqrt(5.0)
    if bc is None:
        bc = [("char", 0.0), ("free",), ("char", 0.5), ("free",), ("char", -0.5), ("free",)]
    faces = []
    for f in range(6):
        xi, side = divmod(f, 2)
        from oracle.elastic import face_slice
        sl = face_slice(xi, side, nodes[xi])
        an = np.sqrt(sum(a[xi][c][sl] ** 2 for c in range(3)))
        faces.append((sl, [a[xi][c][sl] / an for c in range(3)]))

    def exact(t):
        v, s = _plane_wave(kind, X, t, rho, lam, mu, dvec, pol, wl)
        return np.stack(v + s)

    def L(Q, t):
        Qe = exact(t)

        def data(f):
            sl, nvec = faces[f]
            s = [Qe[3 + c][sl] for c in range(6)]
            from oracle.elastic import traction
            return [Qe[c][sl] for c in range(3)], traction(s, nvec)
        return rhs(Q, sch, J, a, mat, bc, data)
    c = math.sqrt((lam + 2 * mu) / rho)
    dt = 0.25 / n / c
    nsteps = int(round(T / dt))
    dt = T / nsteps
    Q = exact(0.0)
    dQ = np.zeros_like(Q)
    for k in range(nsteps):
        rk.rk_step(Q, dQ, k * dt, dt, L)
    err = Q - exact(T)
    W = sch.weights3()
    return math.sqrt(float(np.sum(W * err ** 2)))


@pytest.mark.parametrize("order,kind,lo", [(2, "P", 1.8), (4, "S", 2.8), (6, "P", 3.6),
                                          (3, "S", 2.2), (5, "P", 3.2), (7, "S", 4.0)])
def test_plane_wave_convergence_absorbing_faces(order, kind, lo):
    """Section 6.1 (truncation error structure and the a-priori error estimate): with
    boundary data from the exact plane wave on all six faces, absorbing penalty
    (gamma = 0), the H-norm error on a curvilinear mesh converges at least at the
    global order p + 1 = 2, 3, 4 (closure accuracy p = floor(order/2); the odd orders 3, 5,
    7 measure 2.41, 3.46, 4.31 between n = 16 and 32)."""
    e1 = _mms_error(order, 16, kind, bc=[("char", 0.0)] * 6)
    e2 = _mms_error(order, 32, kind, bc=[("char", 0.0)] * 6)
    rate = math.log2(e1 / e2)
    assert rate > lo, (e1, e2, rate)


@pytest.mark.parametrize("order,kind,lo", [(2, "P", 1.4), (4, "S", 2.25), (6, "P", 3.2),
                                          (3, "S", 1.3), (5, "P", 2.1), (7, "S", 3.4)])
def test_plane_wave_convergence_with_free_surfaces(order, kind, lo):
    """Same with three free-surface faces and gamma = 0, 0.5, -0.5 on the others.  The
    energy-conserving free-surface penalty adds no boundary dissipation, and the
    observed rate is the p + 1/2 that Theorem (error estimate) guarantees for an O(h^p)
    boundary truncation error on a layer of width O(h).  The odd orders 3, 5, 7 measure
    1.44, 2.34, 3.72 between n = 16 and 32: orders 3 and 5 still below p + 1/2 there."""
    e1 = _mms_error(order, 16, kind)
    e2 = _mms_error(order, 32, kind)
    rate = math.log2(e1 / e2)
    assert rate > lo, (e1, e2, rate)


def _interior_truncation(order, n, kind, mapname, ext=1.0, medium=(1.0, 2.0, 1.0), wl=0.8, operator="upwind"):
    """max |dQ/dt_h(Q) - dQ/dt| / max |dQ/dt| for the exact plane wave of _plane_wave at t = 0,
    over the nodes at least b + max(r, q) from every face: there every row is the interior
    stencil of Table 1 applied to metrics formed by interior rows (the closure rows, their
    stencil reach and the penalised face nodes are left out)."""
    nodes = (n + 1, n + 1, n + 1)
    fmap = make_map("curvy", (ext,) * 3, eps=0.05) if mapname == "curvy" else make_map("identity", (ext,) * 3)
    X = node_coordinates(fmap, nodes)
    J, a = metrics(*X, order)
    rho, lam, mu = medium
    mat = tuple(np.full(J.shape, v) for v in (rho, lam, mu))
    dvec = np.array([1.0, 2.0, 2.0]) / 3.0
    pol = dvec if kind == "P" else np.array([2.0, -1.0, 0.0]) / math.sqrt(5.0)
    v, s = _plane_wave(kind, X, 0.0, rho, lam, mu, dvec, pol, wl)
    # time derivative in closed form: d/dt F'(d.x - c t) = -c F''(d.x - c t), F'' = -k^2 sin
    c = math.sqrt((lam + 2 * mu) / rho) if kind == "P" else math.sqrt(mu / rho)
    k = 2 * math.pi / wl
    F2 = -k * k * np.sin(k * (dvec[0] * X[0] + dvec[1] * X[1] + dvec[2] * X[2]))
    E = 0.5 * (np.outer(pol, dvec) + np.outer(dvec, pol))
    S = lam * np.trace(E) * np.eye(3) + 2 * mu * E
    Sv = (S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2])
    Qt = np.stack([c * c * pol[i] * F2 for i in range(3)] + [-c * sv * F2 for sv in Sv])
    R = rhs(np.stack(v + s), Scheme(order, nodes, operator), J, a, mat, [("char", 0.0)] * 6)
    if operator == "upwind":
        r, q, _ = TABLE1[order]
        m = CLOSURE[order]["b"] + max(r, q)
    else:
        m = TRADITIONAL[order]["b"] + order // 2
    inner = (slice(None),) + (slice(m, n + 1 - m),) * 3
    return np.abs(R - Qt)[inner].max() / np.abs(Qt).max()


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("kind", ["P", "S"])
def test_interior_truncation_error_at_design_order(order, kind):
    """Interior accuracy 2p (Table 1, Eq. acc): on the Cartesian grid (exact metrics) the
    local truncation error of the whole right-hand side for an oblique plane wave, which
    exercises the stencils along q, r and s together with the flux and strain forms, falls as
    h^(2p) away from the faces (measured 1.99, 3.99, 5.99 between n = 24 and 48)."""
    e1 = _interior_truncation(order, 24, kind, "identity")
    e2 = _interior_truncation(order, 48, kind, "identity")
    assert math.log2(e1 / e2) > order - 0.1, (e1, e2)


@pytest.mark.parametrize("order", [8, 9])
@pytest.mark.parametrize("kind", ["P", "S"])
def test_interior_truncation_error_orders_8_9(order, kind):
    """The same for orders 8 (Table 1 with alpha_4 = -1/28) and 9: the rows they leave out reach
    13 nodes in from each face, so the grids are n = 32 and 64 (measured slopes 7.98 and
    8.91-8.95)."""
    e1 = _interior_truncation(order, 32, kind, "identity")
    e2 = _interior_truncation(order, 64, kind, "identity")
    assert math.log2(e1 / e2) > order - 0.15, (e1, e2)


@pytest.mark.parametrize("kind", ["P", "S"])
def test_interior_truncation_homogeneous_medium_in_physical_units(kind):
    """The first workload's homogeneous medium (rho = 2700 kg/m^3, vp = 6000 m/s, vs = 3464 m/s)
    on a 1 km cube with an 800 m wavelength: the same relative truncation errors and rate as the
    unit problem, so no step of the scheme depends on the units (order 6)."""
    rho, vp, vs = 2700.0, 6000.0, 3464.0
    med = (rho, rho * (vp * vp - 2 * vs * vs), rho * vs * vs)
    e1 = _interior_truncation(6, 24, kind, "identity", 1000.0, med, 800.0)
    e2 = _interior_truncation(6, 48, kind, "identity", 1000.0, med, 800.0)
    assert math.log2(e1 / e2) > 5.9, (e1, e2)
    u1 = _interior_truncation(6, 24, kind, "identity", 1.0, med, 0.8)
    assert abs(e1 - u1) < 1e-6 * u1, (e1, u1)


@pytest.mark.parametrize("order,lo", [(4, 3.6), (6, 5.0)])
def test_interior_truncation_error_curvilinear(order, lo):
    """Same on the curved map: the metric terms come from D_c = (D+ + D-)/2, whose interior rows
    are of order 2p as well; the observed rate approaches 2p from below as the mesh is refined
    (about 3.8 and 5.2 between n = 32 and 64, 3.9 and 5.7 between 48 and 96)."""
    e1 = _interior_truncation(order, 32, "P", "curvy")
    e2 = _interior_truncation(order, 64, "P", "curvy")
    assert math.log2(e1 / e2) > lo, (e1, e2)


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_pointwise_oracle_matches_whole_array(order):
    nodes = (19, 17, 20)
    fmap = make_map("curvy", (1000.0, 1200.0, 900.0))
    fmed = make_medium("smooth_gradient", Lz=900.0)
    X = node_coordinates(fmap, nodes)
    J, a = metrics(*X, order)
    mat = fmed(*X)
    bc = [("char", 0.0)] * 5 + [("free",)]
    K, Jj, I = np.meshgrid(np.arange(nodes[2]), np.arange(nodes[1]), np.arange(nodes[0]), indexing="ij")

    def fs(i, j, k):
        return smooth_state(nodes, 3, np.asarray(i), np.asarray(j), np.asarray(k))
    R = rhs(np.stack(fs(I, Jj, K)), Scheme(order, nodes), J, a, mat, bc)
    po = PointOracle(order, nodes, fmap, fmed, bc)
    for node in [(0, 0, 0), (18, 16, 19), (5, 7, 19), (9, 8, 10), (3, 0, 12), (18, 3, 0)]:
        got = po.rhs_at(node, fs)
        assert np.abs(got - R[:, node[2], node[1], node[0]]).max() < 1e-13 * np.abs(R).max()


@pytest.mark.parametrize("order,sizes", [(2, (17, 33, 65)), (4, (17, 33, 65)), (6, (33, 65))])
def test_free_stream_residual_converges_at_design_order(order, sizes):
    """A constant state has zero continuous right-hand side (the metric identity
    sum_xi d/dxi (J grad xi) = 0, Sec. 2.2).  The discrete residual (metrics by D_c, flux by
    D-, velocity by D+; no penalties) is not zero on a curved grid, but in the interior it
    falls at the interior order of the operators (free-stream preservation is not enforced)."""
    errs = []
    for n in sizes:
        nodes = (n, n, n)
        x, y, z = node_coordinates(make_map("curvy", (1.0, 1.2, 0.9)), nodes)
        J, a = metrics(x, y, z, order)
        sch = Scheme(order, nodes)
        Q = np.zeros((9,) + x.shape)
        Q[:3] = np.array([0.3, -0.2, 0.5])[:, None, None, None]
        Q[3:] = np.array([1.0, 0.7, -0.4, 0.3, 0.2, -0.5])[:, None, None, None]
        ones = np.ones_like(x)
        rv, e = rhs_raw(Q, sch, a, (ones, ones, ones), [("free",)] * 6, with_sat=False)
        c = (slice(None),) + (slice(n // 4, 3 * n // 4 + 1),) * 3
        errs.append(max(np.abs(np.array(rv)[c]).max(), np.abs(np.array(e)[c]).max()))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > order - 0.3, rates


@pytest.mark.parametrize("geometry,order", [("identity", 4), ("curvy", 4), ("curvy", 6)])
def test_cfl_half_step_lies_inside_the_runge_kutta_stability_limit(geometry, order):
    """dt rho(L) for the dt rule at CFL 0.5 (dt = CFL h_min / c_p,max): the spectral radius of
    the full operator (penalties included) by power iteration in the discrete energy norm,
    in which L is skew-adjoint plus a dissipative part, must stay below 3.34, where the
    scheme's stability region (|R(iy)| <= 1, R the stability polynomial) leaves the
    imaginary axis.  Grid spacing and medium of the 33^3 cube workload."""
    from workloads.timestep import stable_dt
    n, h = 20, 1000.0 / 32
    nodes = (n, n, n)
    X = node_coordinates(make_map(geometry, (h * (n - 1),) * 3), nodes)
    mat = make_medium("homogeneous")(*X)
    J, a = metrics(*X, order)
    sch = Scheme(order, nodes)
    dt = stable_dt(*X, *mat, 0.5)
    bc = [("char", 0.0)] * 5 + [("free",)]
    rng = np.random.default_rng(0)
    Q = rng.normal(size=(9,) + X[0].shape)
    Q[3:] *= 1e7
    Q /= math.sqrt(energy(Q, sch, J, mat))
    lam = 0.0
    for _ in range(250):
        Y = rhs(Q, sch, J, a, mat, bc)
        lam = math.sqrt(energy(Y, sch, J, mat))
        Q = Y / lam
    assert 1.0 < lam * dt < 3.34, lam * dt
    # the limit itself, from the scheme's Butcher tableau: R(z) = 1 + z b^T (I - z A)^-1 1 has
    # |R(iy)| <= 1 up to y = 3.34 and exceeds 1 beyond
    At, bt, _ = rk.butcher_tableau()
    At = np.array(At, dtype=float)
    bt = np.array(bt, dtype=float)

    def R(z):
        return 1.0 + z * bt @ np.linalg.solve(np.eye(len(bt)) - z * At, np.ones(len(bt)))
    assert abs(R(3.30j)) <= 1.0 and abs(R(3.40j)) > 1.0


def test_receivers_record_the_plane_wave_at_their_nodes_after_each_step():
    """The oracle's receivers: traces[n][r][c] is velocity component c at node (i, j, k) of
    receiver r after step n + 1.  On an exact plane wave (P wave along (1, 2, 2)/3, so the
    field varies along every axis) interior receivers must reproduce the exact solution at
    their own node and time to the discretization error; a transposed node index or a
    one-step shift in time misses it by far more."""
    from oracle.solver import OracleSolver
    order, n = 4, 24
    nodes = (n + 1, n + 1, n + 1)
    X = node_coordinates(make_map("curvy", (1.0, 1.0, 1.0), eps=0.05), nodes)
    rho, lam, mu = 1.0, 2.0, 1.0
    mat = tuple(np.full(X[0].shape, v) for v in (rho, lam, mu))
    dvec = np.array([1.0, 2.0, 2.0]) / 3.0
    wl = 0.8

    def exact(t):
        v, s = _plane_wave("P", X, t, rho, lam, mu, dvec, dvec, wl)
        return np.stack(v + s)
    orc = OracleSolver(order, *X, mat, [("char", 0.0)] * 6)
    orc.Q[:] = exact(0.0)
    rec = [(8, 12, 15), (15, 9, 11), (12, 16, 8)]
    orc.receivers = rec
    c = math.sqrt((lam + 2 * mu) / rho)
    dt = 0.25 / n / c
    nsteps = 6
    orc.step(dt, nsteps)
    got = np.array(orc.traces)                          # [step][receiver][component]
    want = np.array([[[exact((s + 1) * dt)[cc][k, j, i] for cc in range(3)] for (i, j, k) in rec]
                     for s in range(nsteps)])
    scale = np.abs(want).max()
    err = np.abs(got - want).max() / scale
    assert err < 5e-3, err
    shifted = np.array([[[exact(s * dt)[cc][k, j, i] for cc in range(3)] for (i, j, k) in rec]
                        for s in range(nsteps)])
    transposed = np.array([[[exact((s + 1) * dt)[cc][i, j, k] for cc in range(3)] for (i, j, k) in rec]
                           for s in range(nsteps)])
    assert np.abs(got - shifted).max() / scale > 10 * err
    assert np.abs(got - transposed).max() / scale > 10 * err
