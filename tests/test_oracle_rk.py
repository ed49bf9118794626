"""Pins of the oracle's 2N-storage RK4 (Carpenter-Kennedy (5,4), cited in Sections 1 and 7)."""
import math
from fractions import Fraction as Fr

import numpy as np

from oracle import rk


def test_classical_order_conditions():
    """The equivalent Butcher tableau satisfies the eight order-4 conditions (to the
    precision of the published rational approximations) and c_i = sum_j a_ij."""
    a, b, c = rk.butcher_tableau()
    a = [[float(x) for x in row] for row in a]
    b = [float(x) for x in b]
    c = [float(x) for x in c]
    s = 5
    assert max(abs(c[i] - float(rk.RK_C[i])) for i in range(s)) < 1e-15
    # the published stage times of the (5,4) scheme, to the digits they agree on
    for ci, pub in zip(rk.C, (0.0, 0.1496590219992291, 0.3704009573642048, 0.6222557631344432, 0.9582821306746903)):
        assert abs(ci - pub) < 1e-12
    cond = [
        (sum(b), 1.0),
        (sum(b[i] * c[i] for i in range(s)), 1 / 2),
        (sum(b[i] * c[i] ** 2 for i in range(s)), 1 / 3),
        (sum(b[i] * a[i][j] * c[j] for i in range(s) for j in range(s)), 1 / 6),
        (sum(b[i] * c[i] ** 3 for i in range(s)), 1 / 4),
        (sum(b[i] * c[i] * a[i][j] * c[j] for i in range(s) for j in range(s)), 1 / 8),
        (sum(b[i] * a[i][j] * c[j] ** 2 for i in range(s) for j in range(s)), 1 / 12),
        (sum(b[i] * a[i][j] * a[j][k] * c[k] for i in range(s) for j in range(s) for k in range(s)), 1 / 24),
    ]
    for got, want in cond:
        assert abs(got - want) < 1e-11, (got, want)


def test_stability_polynomial():
    """R(z) = sum_{k<=4} z^k/k! + z^5/200; |R(iy)| <= 1 up to y ~ 3.34, > 1 beyond 3.36."""
    a, b, c = rk.butcher_tableau()
    A = np.array([[float(x) for x in r] for r in a])
    bb = np.array([float(x) for x in b])
    coef = [1.0] + [bb @ np.linalg.matrix_power(A, k - 1) @ np.ones(5) for k in range(1, 6)]
    for k in range(5):
        assert abs(coef[k] - 1 / math.factorial(k)) < 1e-11
    assert abs(coef[5] - 1 / 200) < 1e-11

    def R(z):
        return sum(coef[k] * z ** k for k in range(6))
    assert all(abs(R(1j * y)) <= 1 + 1e-12 for y in np.linspace(0, 3.34, 400))
    assert abs(R(1j * 3.36)) > 1


def test_observed_fourth_order_nonautonomous():
    """y' = -y + cos(t) sin(3t) y... solved with rk_step; error ratio under halving -> 16."""
    def L(y, t):
        return np.array([-0.5 * y[0] + math.cos(2 * t) * y[1], -math.sin(t) * y[0] - 0.3 * y[1] + math.cos(3 * t)])

    def solve(n):
        y = np.array([1.0, 0.5])
        dy = np.zeros(2)
        t, dt = 0.0, 2.0 / n
        for _ in range(n):
            rk.rk_step(y, dy, t, dt, L)
            t += dt
        return y
    ref = solve(4096)
    errs = [np.abs(solve(n) - ref).max() for n in (16, 32, 64)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.8 < r < 4.6 for r in rates), rates


def test_coefficients_are_fractions():
    assert all(isinstance(x, Fr) for x in rk.RK_A + rk.RK_B + rk.RK_C)
    assert rk.RK_A[0] == 0 and rk.RK_C[0] == 0
