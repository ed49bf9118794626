"""Exact upwind diagonal-norm dual-pair SBP operators (oracle).

Test infrastructure only; see ``oracle/__init__.py``.

Definition (Section 4.1, Eq. upw_SBP and the Definition that follows it): a
triple (H, D-, D+) on n+1 nodes with H diagonal and positive,

    (D+ f)^T H g + f^T H (D- g) = f_n g_n - f_0 g_0       for all f, g,

i.e. H D+ + D-^T H = B with B = diag(-1, 0, ..., 0, 1), and with
D+ + D+^T negative semi-definite.  Order 2p (Eq. acc and the paragraph after
it): D(xi^m) = m xi^(m-1) for m <= 2p at interior rows and m <= p in the
closure rows.

The paper gives only the interior stencils (Table 1, Section 6.2) and cites
Mattsson (2017) for the closures.  Readings taken here (every one is checked
by tests/test_oracle_operators.py):

* Interior rows of D+ are Table 1's alpha_j at offsets -r..q; interior rows of
  D- use beta_j = -alpha_{-j} (Section 6.2).
* Table 1 prints alpha_4 = 1/28 for order 8; with that sign the stencil is not
  consistent (sum 1/14), with -1/28 every moment up to 8 holds.  The table
  below carries -1/28.
* D- is the mirror image of D+: D- = -J D+ J with J the index reversal, which
  is what beta_j = -alpha_{-j} says inside.
* Write M = H D+ (so D+ = H^-1 M and, from the SBP relation,
  D- = H^-1 (B - M^T)).  M equals the Toeplitz interior stencil everywhere
  except in a b-by-b corner block at each end; the lower-right block follows
  from the upper-left one through M - J M^T J = B.  The unknowns are the
  upper-left block of M and the first b weights of H; the equations are the
  closure-row accuracy conditions of D+ and of D- (degree <= p).
* The solution has free parameters (none for order 2, one for order 4, four
  for order 6 with b = 6).  They are fixed at the simple rationals in
  CLOSURE below, chosen (numerically, once) to keep M + M^T - B negative
  semi-definite and the spectral radius of D+ at the value of the interior
  stencil.  These closures are therefore NOT Mattsson's published ones; they
  satisfy the same defining properties.
* Odd orders 3, 5, 7 (Table 1) take the same construction with closure
  accuracy p = (order - 1)/2 and b = 2, 4, 6: order 3 is unique, order 5 has
  one free entry and order 7 four.  Their norms are forced by accuracy; the
  free entries were again chosen numerically, once, for the smallest spectral
  radius of D+ (N = 60) with H > 0 and M + M^T - B <= 0, then rounded to
  rationals with denominators up to 100 and checked exactly.
* Order 8 (Table 1 with alpha_4 = -1/28) takes b = 8, closure accuracy p = 4.
  The accuracy conditions fix the eight weights and all of M's corner block
  but the 3 x 3 sub-block of rows and columns 5..7, whose nine entries are
  free.  They were chosen by a numerical search (oracle/closure_search.py)
  inside the solution set of the accuracy system (minimise the largest nonzero eigenvalue of
  M + M^T - B, then the spectral radius of D+, with H > 0), rounded to
  denominators up to 10^5 and checked exactly.  Coarser rounding (10^4)
  breaks the semi-definiteness.  Its spectral radius (1.75 at N = 61) sits
  below the interior stencil's 2.10.
* Order 9 (Table 1) takes the same b = 8 and p = 4, with the same nine free
  entries; its search optimum lies on the edge of semi-definiteness, so it
  needs denominators up to 10^6 (10^5 breaks the condition).  Spectral
  radius 1.81 at N = 61 against the interior stencil's 1.85.
"""
from fractions import Fraction as Fr

import numpy as np

# Table 1: interior coefficients alpha_j of D+ (interior order, r, q, alpha_-r..alpha_q).
TABLE1 = {
    2: (0, 2, ("-3/2", "2", "-1/2")),
    3: (1, 2, ("-1/3", "-1/2", "1", "-1/6")),
    4: (1, 3, ("-1/4", "-5/6", "3/2", "-1/2", "1/12")),
    5: (2, 3, ("1/20", "-1/2", "-1/3", "1", "-1/4", "1/30")),
    6: (2, 4, ("1/30", "-2/5", "-7/12", "4/3", "-1/2", "2/15", "-1/60")),
    7: (3, 4, ("-1/105", "1/10", "-3/5", "-1/4", "1", "-3/10", "1/15", "-1/140")),
    8: (3, 5, ("-1/168", "1/14", "-1/2", "-9/20", "5/4", "-1/2", "1/6", "-1/28", "1/280")),
    9: (4, 5, ("1/504", "-1/42", "1/7", "-2/3", "-1/5", "1", "-1/3", "2/21", "-1/56", "1/630")),
}

# Table 2: interior coefficients gamma_1..gamma_q of the traditional central SBP operator.
TABLE2 = {
    2: ("1/2",),
    4: ("2/3", "-1/12"),
    6: ("3/4", "-3/20", "1/60"),
    8: ("4/5", "-1/5", "4/105", "-1/280"),
}

# Closure width b and the chosen values of the free entries of M = H D+ (upper-left block).
CLOSURE = {
    2: dict(b=2, free={}),
    3: dict(b=2, free={}),
    4: dict(b=4, free={(3, 3): Fr(-4, 5)}),
    5: dict(b=4, free={(3, 3): Fr(-3, 8)}),
    6: dict(b=6, free={(4, 4): Fr(-17, 25), (4, 5): Fr(131, 100),
                       (5, 4): Fr(-29, 100), (5, 5): Fr(-3, 5)}),
    7: dict(b=6, free={(4, 4): Fr(-1, 4), (4, 5): Fr(47, 50),
                       (5, 4): Fr(-27, 50), (5, 5): Fr(-1, 4)}),
    8: dict(b=8, free={(5, 5): Fr(-40823, 50000), (5, 6): Fr(61471, 50000),
                       (5, 7): Fr(-41397, 100000), (6, 5): Fr(16959, 100000),
                       (6, 6): Fr(-75619, 100000), (6, 7): Fr(31709, 25000),
                       (7, 5): Fr(-18107, 100000), (7, 6): Fr(-35543, 100000),
                       (7, 7): Fr(-23601, 50000)}),
    9: dict(b=8, free={(5, 5): Fr(-756961, 1000000), (5, 6): Fr(1530357, 1000000),
                       (5, 7): Fr(-54319, 125000), (6, 5): Fr(-36707, 100000),
                       (6, 6): Fr(-519783, 1000000), (6, 7): Fr(132041, 125000),
                       (7, 5): Fr(658, 15625), (7, 6): Fr(-565103, 1000000),
                       (7, 7): Fr(-219601, 1000000)}),
}


def interior_stencil(order):
    """alpha_j of Table 1 as {offset j: Fraction}."""
    r, q, coeffs = TABLE1[order]
    return {j: Fr(c) for j, c in zip(range(-r, q + 1), coeffs)}


def interior_stencil_minus(order):
    """beta_j = -alpha_{-j}, the interior stencil of D- (Section 6.2)."""
    return {-j: -a for j, a in interior_stencil(order).items()}


def _solve_exact(rows, rhs, nunk):
    """Solve the linear system rows @ u = rhs exactly (Fractions, Gauss-Jordan).

    Raises ValueError when the system is inconsistent or leaves unknowns free.
    """
    A = [list(r) + [b] for r, b in zip(rows, rhs)]
    piv_cols = []
    row = 0
    for col in range(nunk):
        pr = next((i for i in range(row, len(A)) if A[i][col] != 0), None)
        if pr is None:
            continue
        A[row], A[pr] = A[pr], A[row]
        p = A[row][col]
        A[row] = [x / p for x in A[row]]
        for i in range(len(A)):
            if i != row and A[i][col] != 0:
                f = A[i][col]
                A[i] = [x - f * y for x, y in zip(A[i], A[row])]
        piv_cols.append(col)
        row += 1
    if any(all(x == 0 for x in A[i][:nunk]) and A[i][nunk] != 0 for i in range(len(A))):
        raise ValueError("inconsistent closure system")
    if len(piv_cols) != nunk:
        raise ValueError(f"closure system leaves {nunk - len(piv_cols)} unknowns free")
    u = [Fr(0)] * nunk
    for i, col in enumerate(piv_cols):
        u[col] = A[i][nunk]
    return u


def _accuracy_system(alpha, b, p):
    """Linear equations on the unknowns Mc[i][j] (index i b + j) and w_i (index b b + i): for
    closure rows i < b and degrees m = 0..p, on unit spacing xi_j = j,
      D+ rows:  sum_j M[i, j] j^m            = m w_i i^(m-1)
      D- rows:  sum_j (B - M^T)[i, j] j^m    = m w_i i^(m-1)
    with M equal to the Toeplitz stencil alpha outside the b x b corner block."""
    nunk = b * b + b

    def mi(i, j):
        return i * b + j

    def wi(i):
        return b * b + i

    rows, rhs = [], []
    for i in range(b):
        for m in range(p + 1):
            # D+ accuracy at row i
            row = [Fr(0)] * nunk
            const = Fr(0)
            for j in range(b):
                row[mi(i, j)] += Fr(j) ** m
            for j in range(b, i + max(alpha) + 1):
                if j - i in alpha:
                    const += alpha[j - i] * Fr(j) ** m
            if m >= 1:
                row[wi(i)] -= m * Fr(i) ** (m - 1)
            rows.append(row)
            rhs.append(-const)
            # D- accuracy at row i: (B - M^T)[i, j] = B[j, i] - M[j, i]
            row = [Fr(0)] * nunk
            const = Fr(-1) if (i == 0 and m == 0) else Fr(0)
            for j in range(b):
                row[mi(j, i)] -= Fr(j) ** m
            for j in range(b, i - min(alpha) + 1):
                if i - j in alpha:
                    const -= alpha[i - j] * Fr(j) ** m
            if m >= 1:
                row[wi(i)] -= m * Fr(i) ** (m - 1)
            rows.append(row)
            rhs.append(-const)
    return rows, rhs, nunk


def _pin(rows, rhs, b, nunk, free):
    """Append one equation Mc[i][j] = v per entry of `free`."""
    for (i, j), v in free.items():
        row = [Fr(0)] * nunk
        row[i * b + j] = Fr(1)
        rows.append(row)
        rhs.append(v)


def closure(order):
    """Upper-left block Mc (b x b) of M = H D+ and the boundary weights w_0..w_{b-1}.

    Unknowns: Mc[i][j] (i, j < b) and w_i.  Equations: the accuracy conditions of the D+ and
    D- closure rows up to degree p = floor(order/2) (_accuracy_system), plus one equation per
    free parameter of CLOSURE.
    """
    b = CLOSURE[order]["b"]
    rows, rhs, nunk = _accuracy_system(interior_stencil(order), b, order // 2)
    _pin(rows, rhs, b, nunk, CLOSURE[order]["free"])
    u = _solve_exact(rows, rhs, nunk)
    Mc = [[u[i * b + j] for j in range(b)] for i in range(b)]
    w = [u[b * b + i] for i in range(b)]
    return Mc, w


def min_nodes(order):
    """Fewest nodes per axis for which the two closures stay disjoint and every
    closure row of D- reaches only pure-stencil rows of M (N >= 2b + max(r, q))."""
    r, q, _ = TABLE1[order]
    return 2 * CLOSURE[order]["b"] + max(r, q)


def _assemble_exact(alpha, b, Mc, w, N):
    """(H, M, B) on N nodes, unit spacing: M is the Toeplitz stencil alpha with the corner block
    Mc at the upper left and, through M - J M^T J = B, its mirror at the lower right; H holds
    the weights w at both ends and 1 inside."""
    n = N - 1
    M = [[Fr(0)] * N for _ in range(N)]
    for i in range(N):
        for k, a in alpha.items():
            if 0 <= i + k < N:
                M[i][i + k] = a
    Bm = [[Fr(0)] * N for _ in range(N)]
    Bm[0][0] = Fr(-1)
    Bm[n][n] = Fr(1)
    for i in range(b):
        for j in range(b):
            M[i][j] = Mc[i][j]
    for i in range(b):
        for j in range(b):
            M[n - j][n - i] = Mc[i][j] - Bm[i][j]
    H = [Fr(1)] * N
    for i in range(b):
        H[i] = w[i]
        H[n - i] = w[i]
    return H, M, Bm


def upwind_pair_exact(order, N):
    """(H, Dm, Dp, M, B) on N nodes with unit spacing, as lists of Fractions.

    H is the list of diagonal weights.  Dp = H^-1 M, Dm = H^-1 (B - M^T).
    """
    if order not in CLOSURE:
        raise ValueError("closures are built for orders 2 to 9")
    if N < min_nodes(order):
        raise ValueError(f"order {order} needs at least {min_nodes(order)} nodes")
    Mc, w = closure(order)
    H, M, Bm = _assemble_exact(interior_stencil(order), CLOSURE[order]["b"], Mc, w, N)
    Dp = [[M[i][j] / H[i] for j in range(N)] for i in range(N)]
    Dm = [[(Bm[i][j] - M[j][i]) / H[i] for j in range(N)] for i in range(N)]
    return H, Dm, Dp, M, Bm


def upwind_pair(order, N, length=1.0):
    """Float64 (H, Dm, Dp) on N nodes spanning [0, length]: spacing h = length/(N-1).

    Dm and Dp are scipy CSR matrices.  D+- scale as 1/h and H as h
    (Section 4.1).  Rows b..N-1-b are Table 1's stencils (alpha_j for D+,
    beta_j = -alpha_{-j} for D-); the b closure rows at each end are taken
    from the exact operator on min_nodes(order) nodes, whose left rows do not
    depend on N and whose right rows are the mirror images
    D+[N-1-i, N-1-j] = -D-[i, j] (tests check this against
    upwind_pair_exact for several N).
    """
    import scipy.sparse as sps
    if N < min_nodes(order):
        raise ValueError(f"order {order} needs at least {min_nodes(order)} nodes")
    b = CLOSURE[order]["b"]
    H0, Dm0, Dp0, _, _ = upwind_pair_exact(order, min_nodes(order))
    alpha = interior_stencil(order)
    beta = interior_stencil_minus(order)
    h = length / (N - 1)
    rows = {"p": ([], [], []), "m": ([], [], [])}
    for name, D0, Dother0, st in (("p", Dp0, Dm0, alpha), ("m", Dm0, Dp0, beta)):
        ri, ci, vi = rows[name]
        for i in range(N):
            if i < b:
                ent = [(j, D0[i][j]) for j in range(len(D0)) if D0[i][j] != 0]
            elif i > N - 1 - b:
                ii = N - 1 - i
                ent = [(N - 1 - j, -Dother0[ii][j]) for j in range(len(Dother0)) if Dother0[ii][j] != 0]
            else:
                ent = [(i + k, a) for k, a in st.items()]
            for j, a in ent:
                ri.append(i)
                ci.append(j)
                vi.append(float(a) / h)
    Dp = sps.csr_matrix((rows["p"][2], (rows["p"][0], rows["p"][1])), shape=(N, N))
    Dm = sps.csr_matrix((rows["m"][2], (rows["m"][0], rows["m"][1])), shape=(N, N))
    Hf = np.ones(N)
    for i in range(b):
        Hf[i] = float(H0[i])
        Hf[N - 1 - i] = float(H0[i])
    return Hf * h, Dm, Dp


# Traditional (central) diagonal-norm SBP operators of Table 2: closure width b and the chosen
# values of the free entries of M = H D (upper-left block).  Order 8 (b = 8, boundary accuracy 4)
# leaves three entries free and forces the norm; they were chosen (oracle/closure_search.py)
# where the spectral radius of D stays at the interior stencil's 1.73 for N = 20 to 101.  That
# radius is sensitive to them (rounding to denominators of 100 gives 2 to 4.6), hence 500.
TRADITIONAL = {
    2: dict(b=1, free={}),
    4: dict(b=4, free={}),
    6: dict(b=6, free={(4, 2): Fr(-1, 10)}),
    8: dict(b=8, free={(6, 5): Fr(-299, 500), (7, 5): Fr(41, 500), (7, 6): Fr(-187, 250)}),
}


def traditional_stencil(order):
    """Table 2 as a stencil {offset j: coefficient}: (D f)_i = sum_j gamma_j (f_{i+j} - f_{i-j})."""
    st = {0: Fr(0)}
    for j, c in enumerate(TABLE2[order], start=1):
        st[j] = Fr(c)
        st[-j] = -Fr(c)
    return st


def traditional_closure(order):
    """Upper-left block Mc (b x b) of M = H D and the weights w_0..w_{b-1} of the traditional
    operator.

    A central operator is the case D- = D+ = D of the construction above, which asks for
    M + M^T = B (then H D + D^T H = B, Section 4.1).  Inside, and across the edge of the corner
    block, the antisymmetric stencil already gives M + M^T = 0, so the conditions are the
    accuracy equations of _accuracy_system with Table 2's stencil (degree <= floor(order/2)),
    Mc + Mc^T = diag(-1, 0, ..., 0), and one equation per free entry of TRADITIONAL.
    """
    b = TRADITIONAL[order]["b"]
    rows, rhs, nunk = _accuracy_system(traditional_stencil(order), b, order // 2)
    for i in range(b):
        for j in range(i, b):
            row = [Fr(0)] * nunk
            row[i * b + j] += 1
            row[j * b + i] += 1
            rows.append(row)
            rhs.append(Fr(-1) if i == j == 0 else Fr(0))
    _pin(rows, rhs, b, nunk, TRADITIONAL[order]["free"])
    u = _solve_exact(rows, rhs, nunk)
    Mc = [[u[i * b + j] for j in range(b)] for i in range(b)]
    w = [u[b * b + i] for i in range(b)]
    return Mc, w


def traditional_min_nodes(order):
    """Fewest nodes per axis with disjoint closures (N >= 2b + order/2)."""
    return 2 * TRADITIONAL[order]["b"] + order // 2


def traditional_exact(order, N):
    """(H, D, M, B) of the traditional operator on N nodes, unit spacing, as Fractions:
    D = H^-1 M with M + M^T = B."""
    if order not in TRADITIONAL:
        raise ValueError("traditional closures are built for orders 2, 4, 6, 8")
    if N < traditional_min_nodes(order):
        raise ValueError(f"order {order} needs at least {traditional_min_nodes(order)} nodes")
    Mc, w = traditional_closure(order)
    H, M, Bm = _assemble_exact(traditional_stencil(order), TRADITIONAL[order]["b"], Mc, w, N)
    D = [[M[i][j] / H[i] for j in range(N)] for i in range(N)]
    return H, D, M, Bm


def traditional_op(order, N, length=1.0):
    """Float64 (H, D) of the traditional operator on N nodes spanning [0, length]; D is a scipy
    CSR matrix.  Rows within b of x = 0 come from the exact operator on
    traditional_min_nodes(order) nodes (they do not depend on N), rows within b of the far end
    from the mirror relation D[N-1-i, N-1-j] = -D[i, j], and Table 2's stencil elsewhere."""
    import scipy.sparse as sps
    if N < traditional_min_nodes(order):
        raise ValueError(f"order {order} needs at least {traditional_min_nodes(order)} nodes")
    b = TRADITIONAL[order]["b"]
    H0, D0, _, _ = traditional_exact(order, traditional_min_nodes(order))
    st = traditional_stencil(order)
    h = length / (N - 1)
    ri, ci, vi = [], [], []
    for i in range(N):
        if i < b:
            ent = [(j, D0[i][j]) for j in range(len(D0)) if D0[i][j] != 0]
        elif i > N - 1 - b:
            ii = N - 1 - i
            ent = [(N - 1 - j, -D0[ii][j]) for j in range(len(D0)) if D0[ii][j] != 0]
        else:
            ent = [(i + k, a) for k, a in st.items() if a != 0]
        for j, a in ent:
            ri.append(i)
            ci.append(j)
            vi.append(float(a) / h)
    D = sps.csr_matrix((vi, (ri, ci)), shape=(N, N))
    Hf = np.ones(N)
    for i in range(b):
        Hf[i] = float(H0[i])
        Hf[N - 1 - i] = float(H0[i])
    return Hf * h, D


def dispersion_upwind(order, k):
    """Numerical dispersion relation of the interior upwind stencil, c_s = 1
    (Section 6.2, Eq. dispersion_relation_upwind): |sum_j alpha_j e^{i j k}|."""
    alpha = interior_stencil(order)
    k = np.asarray(k, dtype=float)
    re = sum(float(a) * np.cos(j * k) for j, a in alpha.items())
    im = sum(float(a) * np.sin(j * k) for j, a in alpha.items())
    return np.sqrt(re ** 2 + im ** 2)


def dispersion_traditional(order, k):
    """Eq. dispersion_relation_traditional, c_s = 1: |sum_j 2 gamma_j sin(j k)|."""
    g = [Fr(c) for c in TABLE2[order]]
    k = np.asarray(k, dtype=float)
    return np.abs(sum(2 * float(gj) * np.sin((j + 1) * k) for j, gj in enumerate(g)))
