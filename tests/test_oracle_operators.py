"""Pins of the oracle's upwind SBP operators against what the paper and
mathematics fix (Section 4.1, Section 6.2, Tables 1-2)."""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import operators as op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[int(parts[0])] = [Fr(x) for x in parts[1:]]
    return rows


def _moments(stencil, upto):
    return [sum(a * Fr(j) ** m for j, a in stencil.items()) for m in range(upto + 1)]


def test_table1_matches_print_except_order8_alpha4():
    printed = _read_table("table1_upwind_as_printed.txt")
    for order, row in printed.items():
        r, q = int(row[0]), int(row[1])
        mine = op.interior_stencil(order)
        assert sorted(mine) == list(range(-r, q + 1))
        for j, a in zip(range(-r, q + 1), row[2:]):
            if order == 8 and j == 4:
                assert a == Fr(1, 28) and mine[j] == Fr(-1, 28)
            else:
                assert mine[j] == a


@pytest.mark.parametrize("order", range(2, 10))
def test_table1_consistency_and_order(order):
    """Section 6.2: sum alpha = 0, sum j alpha = 1; order-k stencil exact for xi^m, m <= k."""
    mom = _moments(op.interior_stencil(order), order + 1)
    assert mom[0] == 0 and mom[1] == 1
    for m in range(2, order + 1):
        assert mom[m] == 0, (order, m)
    assert mom[order + 1] != 0          # not exact one degree higher


def test_printed_order8_row_is_inconsistent():
    printed = _read_table("table1_upwind_as_printed.txt")[8]
    st = dict(zip(range(-3, 6), printed[2:]))
    assert _moments(st, 1)[0] == Fr(1, 14)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_table2_consistency(order):
    g = [Fr(c) for c in op.TABLE2[order]]
    printed = _read_table("table2_traditional_as_printed.txt")[order][1:]
    assert g == printed
    assert sum(2 * (j + 1) * gj for j, gj in enumerate(g)) == 1
    # odd moments of the antisymmetric stencil: exact up to degree 'order'
    for m in range(3, order + 1, 2):
        assert sum(2 * gj * Fr(j + 1) ** m for j, gj in enumerate(g)) == 0


def test_minus_stencil_mirror():
    for order in range(2, 10):
        a = op.interior_stencil(order)
        b = op.interior_stencil_minus(order)
        assert all(b[-j] == -a[j] for j in a)
        mom = _moments(b, order)
        assert mom[0] == 0 and mom[1] == 1 and all(x == 0 for x in mom[2:])


def _exact(order, N):
    return op.upwind_pair_exact(order, N)


ORDERS = [2, 3, 4, 5, 6, 7, 8, 9]   # orders 2-7 as the kernels use them; 8 and 9 in the oracle only (Table 1)


@pytest.mark.parametrize("order", ORDERS)
def test_sbp_dual_pair_identity_exact(order):
    """Eq. upw_SBP: H D+ + D-^T H = B exactly in rationals."""
    for N in range(op.min_nodes(order), op.min_nodes(order) + 4):
        H, Dm, Dp, M, B = _exact(order, N)
        for i in range(N):
            for j in range(N):
                assert H[i] * Dp[i][j] + Dm[j][i] * H[j] == B[i][j]


@pytest.mark.parametrize("order", ORDERS)
def test_accuracy_conditions_exact(order):
    """Eq. acc: D xi^m = m xi^(m-1), m <= p everywhere and m <= 2p at interior rows."""
    p = order // 2
    b = op.CLOSURE[order]["b"]
    N = op.min_nodes(order) + 5
    H, Dm, Dp, M, B = _exact(order, N)
    for D in (Dp, Dm):
        for m in range(order + 1):
            for i in range(N):
                lhs = sum(D[i][j] * Fr(j) ** m for j in range(N))
                rhs = m * Fr(i) ** (m - 1) if m >= 1 else 0
                if m <= p or b <= i <= N - 1 - b:
                    assert lhs == rhs, (order, m, i)


@pytest.mark.parametrize("order", ORDERS)
def test_mirror_relation_and_positive_norm(order):
    N = op.min_nodes(order) + 3
    H, Dm, Dp, M, B = _exact(order, N)
    assert all(h > 0 for h in H)
    assert all(H[i] == H[N - 1 - i] for i in range(N))
    for i in range(N):
        for j in range(N):
            assert Dm[i][j] == -Dp[N - 1 - i][N - 1 - j]


def _is_psd_exact(A):
    """Exact positive semi-definiteness test (symmetric Gaussian elimination in rationals)."""
    A = [row[:] for row in A]
    n = len(A)
    for k in range(n):
        if A[k][k] < 0:
            return False
        if A[k][k] == 0:
            if any(A[k][j] != 0 for j in range(k, n)):
                return False
            continue
        for i in range(k + 1, n):
            f = A[i][k] / A[k][k]
            if f != 0:
                for j in range(k, n):
                    A[i][j] -= f * A[k][j]
    return True


@pytest.mark.parametrize("order", ORDERS)
def test_dissipation_negative_semidefinite_exact(order):
    """Definition after Eq. upw_SBP, read as: M + M^T - B <= 0 with M = H D+."""
    for N in (op.min_nodes(order), op.min_nodes(order) + 3):
        H, Dm, Dp, M, B = _exact(order, N)
        S = [[-(M[i][j] + M[j][i] - B[i][j]) for j in range(N)] for i in range(N)]
        assert _is_psd_exact(S)


def test_psd_checker_rejects_indefinite():
    assert not _is_psd_exact([[Fr(1), Fr(2)], [Fr(2), Fr(1)]])
    assert _is_psd_exact([[Fr(1), Fr(1)], [Fr(1), Fr(1)]])


def test_order2_closure_is_unique_and_known_norm():
    Mc, w = op.closure(2)
    assert w == [Fr(1, 4), Fr(5, 4)]
    assert op.CLOSURE[2]["free"] == {}


def test_order4_norm_forced_by_accuracy():
    """With b = 4 the accuracy conditions fix H (only M has a free entry)."""
    _, w = op.closure(4)
    saved = dict(op.CLOSURE[4]["free"])
    try:
        op.CLOSURE[4]["free"] = {(3, 3): Fr(-9, 10)}
        _, w2 = op.closure(4)
    finally:
        op.CLOSURE[4]["free"] = saved
    assert w == w2 == [Fr(49, 144), Fr(61, 48), Fr(41, 48), Fr(149, 144)]


@pytest.mark.parametrize("order", ORDERS)
def test_sparse_builder_equals_exact(order):
    for N in (op.min_nodes(order), op.min_nodes(order) + 1, op.min_nodes(order) + 9):
        H, Dm, Dp, _, _ = _exact(order, N)
        Hf, Dmf, Dpf = op.upwind_pair(order, N, length=float(N - 1))
        assert np.allclose(Dpf.toarray(), [[float(x) for x in r] for r in Dp], rtol=0, atol=1e-15)
        assert np.allclose(Dmf.toarray(), [[float(x) for x in r] for r in Dm], rtol=0, atol=1e-15)
        assert np.allclose(Hf, [float(x) for x in H], rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", ORDERS)
def test_spectral_radius_set_by_interior(order):
    """Our closure choice: the spectral radius of D+ stays at the interior stencil's level."""
    N = 61
    _, Dm, Dp = op.upwind_pair(order, N, length=float(N - 1))
    rho = np.abs(np.linalg.eigvals(Dp.toarray())).max()
    interior = op.dispersion_upwind(order, np.linspace(0, np.pi, 2001)).max()
    assert rho <= interior * 1.01


def test_dispersion_relation_shapes():
    """Section 6.2: orders 2, 4 monotone on [0, pi] with omega(pi) = 4, 8/3; order 6 peaks
    below pi and ends at 32/15; odd orders have a clearly negative slope somewhere;
    traditional operators vanish at pi."""
    k = np.linspace(0, np.pi, 4001)
    for order, end in ((2, 4.0), (4, 8.0 / 3.0), (6, 32.0 / 15.0)):
        w = op.dispersion_upwind(order, k)
        assert abs(w[-1] - end) < 1e-12
    assert np.all(np.diff(op.dispersion_upwind(2, k)) >= -1e-12)
    assert np.all(np.diff(op.dispersion_upwind(4, k)) >= -1e-12)
    w6 = op.dispersion_upwind(6, k)
    assert 2.18 < w6.max() < 2.2 and 2.4 < k[np.argmax(w6)] < 2.7
    for order in (3, 5, 7, 9):
        assert np.diff(op.dispersion_upwind(order, k)).min() < -1e-4
    for order in (2, 4, 6, 8):
        assert abs(op.dispersion_traditional(order, np.pi)) < 1e-12
    # small-k consistency: omega ~ k
    for order in range(2, 10):
        assert abs(op.dispersion_upwind(order, 1e-4) - 1e-4) < 1e-8


def test_symbol_real_part_dissipative():
    """Re(sum alpha_j e^{ijk}) <= 0: the interior D+ is dissipative (D+ + D+^T <= 0)."""
    k = np.linspace(0, 2 * np.pi, 4001)
    for order in range(2, 10):
        a = op.interior_stencil(order)
        re = sum(float(c) * np.cos(j * k) for j, c in a.items())
        assert re.max() <= 1e-12


def test_odd_order_norms_forced_by_accuracy():
    """Odd orders 3, 5, 7 (Table 1) with b = 2, 4, 6: the boundary weights follow from the
    closure-row accuracy conditions alone, whatever the free entries (the same values for
    other choices of them), and order 3 has no free entry."""
    assert op.CLOSURE[3]["free"] == {}
    assert op.closure(3)[1] == [Fr(5, 12), Fr(13, 12)]
    for order, alt in ((5, {(3, 3): Fr(-1, 3)}), (7, {(4, 4): Fr(-27, 100), (4, 5): Fr(91, 100),
                                                      (5, 4): Fr(-51, 100), (5, 5): Fr(-1, 4)})):
        w = op.closure(order)[1]
        saved = op.CLOSURE[order]["free"]
        try:
            op.CLOSURE[order]["free"] = alt
            assert op.closure(order)[1] == w
        finally:
            op.CLOSURE[order]["free"] = saved
        # H integrates constants exactly on unit spacing: the b weights add up to b - 1/2
        assert sum(w) == len(w) - Fr(1, 2)


def test_group_velocity_and_spurious_modes():
    """Section 6.2's observations on d omega / dk (negative slope = a spurious unresolved mode
    travelling the wrong way), from Table 1 and Table 2:
    * upwind orders 2 and 4: d omega/dk >= 0 on [0, pi]; order 6 nearly so (minimum -0.15,
      near k = 0.9 pi);
    * odd upwind orders 3, 5, 7, 9 and order 8: clearly negative somewhere (minimum <= -0.2);
    * traditional orders 2 to 8: d omega/dk down to -1 or below, negative on 35-50 % of the
      spectrum (exactly half for order 2, omega = sin k)."""
    k = np.linspace(0, np.pi, 200001)
    dk = k[1] - k[0]

    def min_slope(w):
        return (np.diff(w) / dk).min()
    assert min_slope(op.dispersion_upwind(2, k)) >= -1e-9
    assert min_slope(op.dispersion_upwind(4, k)) >= -1e-9
    assert -0.2 < min_slope(op.dispersion_upwind(6, k)) < 0
    for order in (3, 5, 7, 8, 9):
        assert min_slope(op.dispersion_upwind(order, k)) < -0.2, order
    for order in (2, 4, 6, 8):
        w = op.dispersion_traditional(order, k)
        frac = np.mean(np.diff(w) < 0)
        assert min_slope(w) <= -1 + 1e-6 and 0.35 <= frac <= 0.5 + 1e-9, (order, frac)
    assert abs(np.mean(np.diff(op.dispersion_traditional(2, k)) < 0) - 0.5) < 1e-4


@pytest.mark.parametrize("order", [8, 9])
def test_order8_9_closure_norms_forced(order):
    """Orders 8 and 9 with b = 8: the weights follow from the closure-row accuracy conditions
    alone (other values of the nine free entries give the same ones), integrate constants
    exactly (sum b - 1/2), and every free entry lies in the 3 x 3 block of rows and columns
    5..7.  Order 10 is refused."""
    w = op.closure(order)[1]
    assert sum(w) == 8 - Fr(1, 2) and min(w) > 0
    assert set(op.CLOSURE[order]["free"]) == {(i, j) for i in range(5, 8) for j in range(5, 8)}
    saved = op.CLOSURE[order]["free"]
    try:
        op.CLOSURE[order]["free"] = {k: Fr(0) for k in saved}
        assert op.closure(order)[1] == w
    finally:
        op.CLOSURE[order]["free"] = saved
    with pytest.raises(ValueError):
        op.upwind_pair_exact(10, 40)


def test_order8_closure_needs_the_corrected_table_sign():
    """With alpha_4 = +1/28 as Table 1 prints it the interior stencil is inconsistent, so the
    closure system built on it has no solution for the same free entries."""
    alpha = op.interior_stencil(8)
    assert alpha[4] == Fr(-1, 28)
    bad = dict(alpha)
    bad[4] = Fr(1, 28)
    assert sum(bad.values()) == Fr(1, 14)
    rows, rhs, nunk = op._accuracy_system(bad, 8, 4)
    op._pin(rows, rhs, 8, nunk, op.CLOSURE[8]["free"])
    with pytest.raises(ValueError, match="inconsistent"):
        op._solve_exact(rows, rhs, nunk)


def test_closure_search_rounding_check_accepts_the_tables_and_rejects_a_coarse_rounding():
    """oracle/closure_search.py (how the order-8 and 9 entries were chosen): its exact check
    accepts the tables' entries and rejects order 8's entries rounded to 10^-4, the rounding that
    breaks semi-definiteness; the free entries it finds are the 3 x 3 block of rows 5..7."""
    from oracle import closure_search as cs
    for order, den in ((8, 100000), (9, 1000000)):
        vals = {ij: float(v) for ij, v in op.CLOSURE[order]["free"].items()}
        assert set(cs._free_entries(op.interior_stencil(order), 8, 4)) == set(vals)
        [(d, fr, ok, rho)] = cs.round_upwind(order, vals, [den])
        assert ok and fr == op.CLOSURE[order]["free"] and rho < 1.85
    vals8 = {ij: float(v) for ij, v in op.CLOSURE[8]["free"].items()}
    [(_, _, ok, _)] = cs.round_upwind(8, vals8, [10000])
    assert not ok
