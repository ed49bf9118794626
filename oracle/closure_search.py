"""How the free closure entries of the wide operators in ``oracle/operators.py`` were chosen.

Test infrastructure only, like the rest of ``oracle/``; a design aid that is run by hand and
whose output the CLOSURE and TRADITIONAL tables record:

    python -m oracle.closure_search upwind 8 --trials 4 --dens 10000,100000
    python -m oracle.closure_search upwind 9 --trials 24 --dens 100000,1000000
    python -m oracle.closure_search traditional 8 --trials 12 --dens 100,250,500,1000

Upwind orders 8 and 9 (Section 4.1, Table 1; b = 8, closure accuracy p = 4).  The accuracy
conditions (``operators._accuracy_system``) fix the norm and all but nine entries of the corner
block of M = H D+.  The search works in the solution set of that linear system (a particular
solution plus its null space, in floating point): Powell's method, from the origin and from
seeded random points, first minimises the largest eigenvalue of M + M^T - B other than the zero
of the constant mode (driving it to <= 0, the semi-definiteness reading of Section 4.1), then
that plus the spectral radius of D+ on 64 nodes.  The best point with a negative second
eigenvalue is rounded to rationals of the given denominators; each rounding is re-solved exactly
and accepted only if -(M + M^T - B) is positive semi-definite exactly (rational elimination) on
min_nodes and min_nodes + 3 nodes with H > 0.  The search optimum lies on the edge of
semi-definiteness, so coarse roundings fail.

Traditional order 8 (Table 2; b = 8, p = 4, M + M^T = B imposed): three entries stay free and
the norm is forced.  Nelder-Mead minimises the spectral radius of D on 61 nodes from the origin
and seeded random points; the end points lie along a flat valley (radius 1.721-1.726), and the
radius is very sensitive to rounding, so the roundings of every end point are listed by radius
(the table holds trial 6's rounding to denominator 500).
"""
import argparse
from fractions import Fraction as Fr

import numpy as np

from . import operators as op


def _null_space(alpha, b, p):
    rows, rhs, _ = op._accuracy_system(alpha, b, p)
    A = np.array([[float(x) for x in r] for r in rows])
    y = np.array([float(x) for x in rhs])
    u0 = np.linalg.lstsq(A, y, rcond=None)[0]
    _, sv, Vt = np.linalg.svd(A)
    rank = int((sv > 1e-10 * sv[0]).sum())
    return u0, Vt[rank:].T


def _assemble_float(alpha, b, u, N):
    """(M, H, B) on N nodes from the unknowns u = (corner block row by row, weights)."""
    Mc = u[:b * b].reshape(b, b)
    w = u[b * b:]
    M = np.zeros((N, N))
    for i in range(N):
        for k, a in alpha.items():
            if 0 <= i + k < N:
                M[i, i + k] = float(a)
    Bm = np.zeros((N, N))
    Bm[0, 0], Bm[-1, -1] = -1.0, 1.0
    M[:b, :b] = Mc
    n = N - 1
    for i in range(b):
        for j in range(b):
            M[n - j, n - i] = Mc[i, j] - Bm[i, j]
    H = np.ones(N)
    H[:b] = w
    H[n - b + 1:] = w[::-1]
    return M, H, Bm


def _free_entries(alpha, b, p):
    """The corner-block entries left free by the accuracy system (non-pivot columns)."""
    rows, rhs, nunk = op._accuracy_system(alpha, b, p)
    R = [list(r) for r in rows]
    piv, row = [], 0
    for col in range(nunk):
        pr = next((i for i in range(row, len(R)) if R[i][col] != 0), None)
        if pr is None:
            continue
        R[row], R[pr] = R[pr], R[row]
        pv = R[row][col]
        R[row] = [x / pv for x in R[row]]
        for i in range(len(R)):
            if i != row and R[i][col] != 0:
                f = R[i][col]
                R[i] = [x - f * y for x, y in zip(R[i], R[row])]
        piv.append(col)
        row += 1
    return [(c // b, c % b) for c in range(nunk) if c not in piv and c < b * b]


def _is_psd_exact(S):
    A = [r[:] for r in S]
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


def search_upwind(order, trials, b=8, N=64, seed=0):
    """Best free-entry values (floats, keyed by corner-block entry) and the spectral radius."""
    from scipy.optimize import minimize
    alpha = op.interior_stencil(order)
    u0, Z = _null_space(alpha, b, order // 2)

    def measures(z):
        M, H, Bm = _assemble_float(alpha, b, u0 + Z @ z, N)
        lam = np.linalg.eigvalsh(M + M.T - Bm)
        rho = np.abs(np.linalg.eigvals(M / H[:, None])).max()
        return H.min(), lam[-1], lam[-2], rho

    def objective(z, wrho):
        hmin, l1, l2, rho = measures(z)
        pen = 1e3 * (0.05 - hmin) if hmin <= 0.05 else 0.0
        return l2 * 1e3 + wrho * rho + pen + 1e3 * max(0.0, l1 - 1e-12)

    rng = np.random.default_rng(seed)
    best = None
    for t in range(trials):
        z = rng.normal(scale=0.5, size=Z.shape[1]) if t else np.zeros(Z.shape[1])
        for wrho in (0.0, 1.0):
            z = minimize(objective, z, args=(wrho,), method="Powell",
                         options=dict(maxiter=20000, xtol=1e-6, ftol=1e-10)).x
        hmin, l1, l2, rho = measures(z)
        print(f"trial {t}: min H {hmin:.3f}, eigenvalues {l1:.2e} {l2:.2e}, spectral radius {rho:.3f}")
        if l2 < 0 and hmin > 0 and (best is None or rho < best[1]):
            best = (z, rho)
    if best is None:
        return None, None
    u = u0 + Z @ best[0]
    return {ij: float(u[ij[0] * b + ij[1]]) for ij in _free_entries(alpha, b, order // 2)}, best[1]


def round_upwind(order, values, dens, b=8):
    """For each denominator: the rounded entries, whether they pass the exact checks, and the
    spectral radius of D+ on 61 nodes."""
    alpha = op.interior_stencil(order)
    rows0, rhs0, nunk = op._accuracy_system(alpha, b, order // 2)
    nmin = 2 * b + max(op.TABLE1[order][0], op.TABLE1[order][1])
    out = []
    for den in dens:
        fr = {ij: Fr(round(v * den), den) for ij, v in values.items()}
        rows, rhs = [list(x) for x in rows0], list(rhs0)
        op._pin(rows, rhs, b, nunk, fr)
        u = op._solve_exact(rows, rhs, nunk)
        Mc = [[u[i * b + j] for j in range(b)] for i in range(b)]
        w = [u[b * b + i] for i in range(b)]
        ok = min(w) > 0
        for N in (nmin, nmin + 3):
            H, M, Bm = op._assemble_exact(alpha, b, Mc, w, N)
            ok = ok and _is_psd_exact([[-(M[i][j] + M[j][i] - Bm[i][j]) for j in range(N)] for i in range(N)])
        H, M, _ = op._assemble_exact(alpha, b, Mc, w, 61)
        D = np.array([[float(x) for x in r] for r in M]) / np.array([float(x) for x in H])[:, None]
        out.append((den, fr, ok, float(np.abs(np.linalg.eigvals(D)).max())))
    return out


def search_traditional8(trials, N=61, seed=0):
    """Best three free entries of the traditional order-8 corner block, by spectral radius."""
    from scipy.optimize import minimize
    free = [(6, 5), (7, 5), (7, 6)]
    alpha = op.traditional_stencil(8)
    saved = op.TRADITIONAL[8]["free"]

    def solve(vals):
        op.TRADITIONAL[8]["free"] = dict(zip(free, vals))
        return op.traditional_closure(8)
    try:   # the corner block is affine in the three entries: three exact solves span it
        Mc0, w0 = solve([Fr(0)] * 3)
        basis = []
        for k in range(3):
            v = [Fr(0)] * 3
            v[k] = Fr(1)
            Mck = solve(v)[0]
            basis.append(np.array([[float(Mck[i][j] - Mc0[i][j]) for j in range(8)] for i in range(8)]))
    finally:
        op.TRADITIONAL[8]["free"] = saved
    u0 = np.concatenate([np.array([[float(x) for x in r] for r in Mc0]).ravel(), [float(x) for x in w0]])

    def rho(z):
        u = u0.copy()
        u[:64] += sum(zk * Bk.ravel() for zk, Bk in zip(z, basis))
        M, H, _ = _assemble_float(alpha, 8, u, N)
        return np.abs(np.linalg.eigvals(M / H[:, None])).max()

    rng = np.random.default_rng(seed)
    ends = []
    for t in range(trials):
        z0 = rng.normal(scale=0.5, size=3) if t else np.zeros(3)
        r = minimize(rho, z0, method="Nelder-Mead", options=dict(xatol=1e-6, fatol=1e-9, maxiter=3000))
        print(f"trial {t}: {np.round(r.x, 5)} spectral radius {r.fun:.5f}")
        ends.append((dict(zip(free, r.x)), float(r.fun)))
    return ends, rho


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("family", choices=("upwind", "traditional"))
    ap.add_argument("order", type=int)
    ap.add_argument("--trials", type=int, default=8)
    ap.add_argument("--dens", default="100,1000,10000,100000,1000000")
    a = ap.parse_args()
    dens = [int(x) for x in a.dens.split(",")]
    k = np.linspace(0, np.pi, 4001)
    if a.family == "upwind":
        vals, rho = search_upwind(a.order, a.trials)
        if vals is None:
            print("no semi-definite point found")
            return
        print(f"best spectral radius {rho:.4f}, interior symbol {op.dispersion_upwind(a.order, k).max():.4f}")
        for den, fr, ok, r61 in round_upwind(a.order, vals, dens):
            print(den, "semi-definite" if ok else "NOT semi-definite", f"radius {r61:.4f}",
                  {ij: str(v) for ij, v in fr.items()} if ok else "")
    else:
        if a.order != 8:
            raise SystemExit("the search covers traditional order 8")
        # the end points lie along a flat valley of the radius; roundings of each are compared
        ends, rho_of = search_traditional8(a.trials)
        print(f"interior symbol {op.dispersion_traditional(8, k).max():.4f}")
        for t, (vals, r) in enumerate(ends):
            for den in dens:
                fr = {ij: Fr(round(v * den), den) for ij, v in vals.items()}
                z = np.array([float(v) for v in fr.values()])
                print(f"trial {t} ({r:.4f}), denominator {den}:", {ij: str(v) for ij, v in fr.items()},
                      f"radius {rho_of(z):.4f}")


if __name__ == "__main__":
    main()
