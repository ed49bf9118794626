"""Pins of the oracle's moment-tensor point source (Section 7.1, Eq. momententor_pointsource)."""
import math

import numpy as np
import pytest

from oracle.elastic import Scheme
from oracle.metrics import metrics
from oracle.source import PointSource, delta_weights_1d, loh1_stf, moment_tensor, ricker
from workloads.geometry import make_map, node_coordinates


@pytest.mark.parametrize("xi0,N,m", [(0.37, 33, 5), (0.02, 33, 7), (0.99, 17, 3), (0.5, 97, 7)])
def test_delta_moment_conditions(xi0, N, m):
    c, phi = delta_weights_1d(xi0, N, m)
    h = 1.0 / (N - 1)
    xs = (np.arange(c, c + m + 1) * h - xi0) / h
    for k in range(m + 1):
        assert abs(np.dot(phi, xs ** k) - (1.0 if k == 0 else 0.0)) < 1e-10
    assert 0 <= c and c + m <= N - 1


def test_discrete_delta_integrates_polynomials_exactly():
    """sum H J delta_h f = f(x_s) for f a polynomial of degree <= order+1 in (q, r, s)."""
    order, nodes = 4, (21, 22, 23)
    X = node_coordinates(make_map("curvy", (1.0, 1.0, 1.0)), nodes)
    J, _ = metrics(*X, order)
    sch = Scheme(order, nodes)
    W = sch.weights3()
    src = PointSource((0.41, 0.57, 0.33), np.zeros(6), lambda t: 0.0, order, nodes, W, J)
    nq, nr, ns = nodes
    q = np.arange(nq)[None, None, :] / (nq - 1)
    r = np.arange(nr)[None, :, None] / (nr - 1)
    s = np.arange(ns)[:, None, None] / (ns - 1)
    f = (1 + 2 * q - q ** 3 + 0.5 * q ** 5) * (2 - r + r ** 4) * (1 + s ** 2 - 0.3 * s ** 5) + 0 * W
    val = np.sum(W[src.sl] * J[src.sl] * src.delta * f[src.sl])
    q0, r0, s0 = 0.41, 0.57, 0.33
    want = (1 + 2 * q0 - q0 ** 3 + 0.5 * q0 ** 5) * (2 - r0 + r0 ** 4) * (1 + s0 ** 2 - 0.3 * s0 ** 5)
    assert abs(val - want) < 1e-10
    assert abs(np.sum(W[src.sl] * J[src.sl] * src.delta) - 1.0) < 1e-12


def test_double_couple_moment_tensor():
    rng = np.random.default_rng(0)
    for _ in range(10):
        st, dp, rk_ = rng.uniform(0, 2 * math.pi), rng.uniform(0.1, math.pi / 2), rng.uniform(-math.pi, math.pi)
        Mv = moment_tensor(st, dp, rk_, 2.0)
        M = np.array([[Mv[0], Mv[3], Mv[4]], [Mv[3], Mv[1], Mv[5]], [Mv[4], Mv[5], Mv[2]]])
        ev = np.sort(np.linalg.eigvalsh(M))
        assert np.allclose(ev, [-2.0, 0.0, 2.0], atol=1e-12)
    # vertical strike-slip on a north-south fault: only M_xy (east-north) is non-zero
    Mv = moment_tensor(0.0, math.pi / 2, 0.0, 1.0)
    assert np.allclose(Mv, [0, 0, 0, 1.0, 0, 0], atol=1e-15)


def test_source_time_functions():
    ts = np.linspace(0, 5, 200001)
    g = np.array([loh1_stf(t) for t in ts])
    assert abs(np.trapezoid(g, ts) - 1.0) < 1e-6
    r = np.array([ricker(t, 2.0, 0.6) for t in ts])
    assert abs(np.trapezoid(r, ts)) < 1e-6 and abs(ricker(0.6, 2.0, 0.6) - 1.0) < 1e-15
