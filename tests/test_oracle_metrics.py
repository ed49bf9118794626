"""Pins of the oracle's Jacobian and metric terms (Section 2.2)."""
import math

import numpy as np
import pytest

from oracle.metrics import metrics
from workloads.geometry import make_map, node_coordinates
from workloads.configs import config_by_name


def _affine_coords(A, c, nodes):
    nq, nr, ns = nodes
    q = np.arange(nq)[None, None, :] / (nq - 1)
    r = np.arange(nr)[None, :, None] / (nr - 1)
    s = np.arange(ns)[:, None, None] / (ns - 1)
    X = [A[i][0] * q + A[i][1] * r + A[i][2] * s + c[i] for i in range(3)]
    shape = (ns, nr, nq)
    return [np.broadcast_to(x, shape).copy() for x in X]


@pytest.mark.parametrize("order", [2, 4, 6])
def test_identity_map(order):
    nodes = (17, 19, 21)
    x, y, z = node_coordinates(make_map("identity", (1000.0, 1200.0, 900.0)), nodes)
    J, a = metrics(x, y, z, order)
    assert np.allclose(J, 1000.0 * 1200.0 * 900.0, rtol=1e-13)
    want = np.diag([1200.0 * 900.0, 1000.0 * 900.0, 1000.0 * 1200.0])
    for xi in range(3):
        for eta in range(3):
            assert np.allclose(a[xi][eta], want[xi, eta], rtol=1e-13, atol=1e-6)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_affine_map_against_matrix_inverse(order):
    """x = A xi + c: J = det A and a = J A^{-1} (xi_eta = (A^-1)_{xi,eta}), via numpy.linalg."""
    rng = np.random.default_rng(7)
    A = np.eye(3) * 1000.0 + rng.normal(scale=150.0, size=(3, 3))
    nodes = (17, 18, 19)
    x, y, z = _affine_coords(A, [10.0, -5.0, 3.0], nodes)
    J, a = metrics(x, y, z, order)
    assert np.allclose(J, np.linalg.det(A), rtol=1e-12)
    Ainv = np.linalg.inv(A)
    for xi in range(3):
        for eta in range(3):
            assert np.allclose(a[xi][eta] / J, Ainv[xi, eta], rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_polynomial_map_exact_to_closure_order(order):
    """A map of degree p = order/2 in (q, r, s) has exact D_c derivatives at every node, so
    J and the metrics equal those of the analytic Jacobian (inverted with numpy.linalg)."""
    p = order // 2
    nodes = (17, 18, 19)
    nq, nr, ns = nodes
    q = (np.arange(nq) / (nq - 1))[None, None, :]
    r = (np.arange(nr) / (nr - 1))[None, :, None]
    s = (np.arange(ns) / (ns - 1))[:, None, None]
    e = 0.1
    # x = q + e q^p r, y = r + e r^p s, z = s + e s^p q
    X = [q + e * q ** p * r, r + e * r ** p * s, s + e * s ** p * q]
    shape = (ns, nr, nq)
    x, y, z = [np.broadcast_to(v, shape).copy() for v in X]
    J, a = metrics(x, y, z, order)
    Q, R, S = np.broadcast_arrays(q, r, s)
    jac = np.zeros(shape + (3, 3))
    jac[..., 0, 0] = 1 + e * p * Q ** (p - 1) * R
    jac[..., 0, 1] = e * Q ** p
    jac[..., 1, 1] = 1 + e * p * R ** (p - 1) * S
    jac[..., 1, 2] = e * R ** p
    jac[..., 2, 2] = 1 + e * p * S ** (p - 1) * Q
    jac[..., 2, 0] = e * S ** p
    Jx = np.linalg.det(jac)
    inv = np.linalg.inv(jac)
    assert np.allclose(J, Jx, rtol=1e-12)
    for xi in range(3):
        for eta in range(3):
            assert np.allclose(a[xi][eta], Jx * inv[..., xi, eta], rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_metric_convergence_smooth_map(order):
    """Max error of J against the analytic Jacobian falls at least at the closure order p."""
    p = order // 2
    errs = []
    for n in (24, 48):
        nodes = (n + 1, n + 1, n + 1)
        fmap = make_map("curvy", (1.0, 1.0, 1.0), eps=0.08)
        x, y, z = node_coordinates(fmap, nodes)
        J, _ = metrics(x, y, z, order)
        # analytic Jacobian by centred complex-free finite differences of the closed form
        qq = np.arange(n + 1) / n
        Q, R, S = np.meshgrid(qq, qq, qq, indexing="ij")
        Q, R, S = Q.transpose(2, 1, 0), R.transpose(2, 1, 0), S.transpose(2, 1, 0)
        d = 1e-6
        cols = []
        for dq in ((d, 0, 0), (0, d, 0), (0, 0, d)):
            xp = np.array(fmap(Q + dq[0], R + dq[1], S + dq[2]))
            xm = np.array(fmap(Q - dq[0], R - dq[1], S - dq[2]))
            cols.append((xp - xm) / (2 * d))
        jac = np.stack(cols, axis=-1)          # [3 (x,y,z), ..., 3 (q,r,s)]
        Jx = np.linalg.det(np.moveaxis(jac, 0, -2))
        errs.append(np.abs(J - Jx).max())
    rate = math.log2(errs[0] / errs[1])
    assert rate > p - 0.3, (errs, rate)


@pytest.mark.parametrize("name", ["hill129_o6", "topo1025_o6_fp32"])
def test_workload_maps_have_positive_jacobian(name):
    cfg = config_by_name(name)
    nodes = tuple(max(17, (n - 1) // 8 + 1) for n in cfg.nodes)
    x, y, z = node_coordinates(make_map(cfg), nodes)
    J, _ = metrics(x, y, z, cfg.order)
    assert J.min() > 0
