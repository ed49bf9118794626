"""Generate the operator coefficient header used by the CUDA kernels.

Run ``python -m paper_2011_02600_gb300.opgen`` to rewrite
``csrc/sbp_coeffs.h``.  The header is committed; the build does not run
this script.

What it derives (Section 4.1 and Table 1 of Duru, Fung & Williams): for the
interior orders 2 to 7, the upwind dual pair (H, D-, D+) whose interior
rows are Table 1's stencil alpha_j (D+) and its mirror beta_j = -alpha_{-j}
(D-), and whose b closure rows at each end make

  * D+ and D- exact for polynomials of degree <= floor(order/2) in every row, and
  * H D+ + D-^T H = diag(-1, 0, ..., 0, 1)   (the SBP dual-pair relation),

with D- the index-reversed negative of D+.  Writing P = H D+, only the
upper-left b x b block of P and the first b entries of H are unknown.  The
accuracy equations leave free entries (none for orders 2 and 3, one for orders
4 and 5, four for orders 6 and 7); they are pinned to the values in
FREE_ENTRIES, which keep P + P^T - B negative semi-definite and the spectral
radius of D+ small.  The kernels are launched for all six orders and for the
traditional operators of orders 2, 4 and 6 (Table 2); orders 8 and 9 reach 5
nodes, more than the kernels' tile halo of 4, and have no tables here.

This module is independent of any other implementation of the operators in
the repository: it carries its own statement of Table 1 and its own exact
solver.
"""
import os
from fractions import Fraction

# Table 1 rows used by the kernels: (r, q, alpha_{-r}..alpha_{q}).
STENCILS = {
    2: (0, 2, [Fraction(-3, 2), Fraction(2), Fraction(-1, 2)]),
    3: (1, 2, [Fraction(-1, 3), Fraction(-1, 2), Fraction(1), Fraction(-1, 6)]),
    4: (1, 3, [Fraction(-1, 4), Fraction(-5, 6), Fraction(3, 2), Fraction(-1, 2), Fraction(1, 12)]),
    5: (2, 3, [Fraction(1, 20), Fraction(-1, 2), Fraction(-1, 3), Fraction(1), Fraction(-1, 4), Fraction(1, 30)]),
    6: (2, 4, [Fraction(1, 30), Fraction(-2, 5), Fraction(-7, 12), Fraction(4, 3), Fraction(-1, 2),
               Fraction(2, 15), Fraction(-1, 60)]),
    7: (3, 4, [Fraction(-1, 105), Fraction(1, 10), Fraction(-3, 5), Fraction(-1, 4), Fraction(1),
               Fraction(-3, 10), Fraction(1, 15), Fraction(-1, 140)]),
}
BLOCK = {2: 2, 3: 2, 4: 4, 5: 4, 6: 6, 7: 6}
# (row, col) of P = H D+ in the upper-left block -> fixed value
FREE_ENTRIES = {
    2: {},
    3: {},
    4: {(3, 3): Fraction(-4, 5)},
    5: {(3, 3): Fraction(-3, 8)},
    6: {(4, 4): Fraction(-17, 25), (4, 5): Fraction(131, 100), (5, 4): Fraction(-29, 100),
        (5, 5): Fraction(-3, 5)},
    7: {(4, 4): Fraction(-1, 4), (4, 5): Fraction(47, 50), (5, 4): Fraction(-27, 50), (5, 5): Fraction(-1, 4)},
}
ORDERS = (2, 3, 4, 5, 6, 7)

# Table 2 (the traditional central operators): gamma_1..gamma_p, (D f)_i = sum_j gamma_j (f_{i+j} - f_{i-j}).
CENTRAL = {
    2: [Fraction(1, 2)],
    4: [Fraction(2, 3), Fraction(-1, 12)],
    6: [Fraction(3, 4), Fraction(-3, 20), Fraction(1, 60)],
}
CENTRAL_BLOCK = {2: 1, 4: 4, 6: 6}
CENTRAL_FREE = {2: {}, 4: {}, 6: {(4, 2): Fraction(-1, 10)}}
TRADITIONAL = 100   # OpCoef<TRADITIONAL + order>: the traditional operator of that order


def _rref_solve(eqs, names):
    """eqs: list of (dict name->coef, rhs).  Returns dict name->value; raises if not unique."""
    rows = [({k: v for k, v in c.items() if v != 0}, r) for c, r in eqs]
    solution_rows = []
    for name in names:
        piv = next((k for k, (c, _) in enumerate(rows) if c.get(name, 0) != 0), None)
        if piv is None:
            raise ValueError(f"unknown {name} is not determined")
        c, r = rows.pop(piv)
        inv = 1 / c[name]
        c = {k: v * inv for k, v in c.items()}
        r = r * inv
        new_rows = []
        for c2, r2 in rows:
            f = c2.get(name, 0)
            if f:
                c2 = dict(c2)
                for k, v in c.items():
                    c2[k] = c2.get(k, 0) - f * v
                    if c2[k] == 0:
                        del c2[k]
                r2 = r2 - f * r
            new_rows.append((c2, r2))
        rows = new_rows
        solution_rows.append((name, c, r))
    for c, r in rows:
        if any(v != 0 for v in c.values()) or r != 0:
            raise ValueError("overdetermined closure system is inconsistent")
    val = {}
    for name, c, r in reversed(solution_rows):
        val[name] = r - sum(v * val[k] for k, v in c.items() if k != name)
    return val


def derive(order):
    """(b, r, q, alpha dict, H weights w[0..b-1], Dplus rows [b][b+q], Dminus rows [b][b+q]).

    order > TRADITIONAL: the traditional operator of order - TRADITIONAL (Table 2), the case
    D- = D+ = D: its antisymmetric stencil, and P + P^T = B on the corner block added to the
    accuracy equations (then H D + D^T H = B)."""
    central = order > TRADITIONAL
    if central:
        o = order - TRADITIONAL
        r = q = o // 2
        alpha = {0: Fraction(0)}
        for j, g in enumerate(CENTRAL[o], start=1):
            alpha[j], alpha[-j] = g, -g
        b, p, free = CENTRAL_BLOCK[o], o // 2, CENTRAL_FREE[o]
    else:
        r, q, coeffs = STENCILS[order]
        alpha = {j: a for j, a in zip(range(-r, q + 1), coeffs)}
        b, p, free = BLOCK[order], order // 2, FREE_ENTRIES[order]
    P = {(i, j): f"P{i}_{j}" for i in range(b) for j in range(b)}
    W = [f"w{i}" for i in range(b)]

    def P_entry(i, j):
        """(unknown name or None, known value) of P[i][j] for i or j < b on a long grid."""
        if i < b and j < b:
            return P[(i, j)], Fraction(0)
        return None, alpha.get(j - i, Fraction(0))

    eqs = []
    for i in range(b):
        for m in range(p + 1):
            target = {W[i]: -m * Fraction(i) ** (m - 1)} if m >= 1 else {}
            # D+ : sum_j P[i][j] j^m - m w_i i^(m-1) = 0
            c, known = dict(target), Fraction(0)
            for j in range(0, b + q + 1):
                name, val = P_entry(i, j)
                if name:
                    c[name] = c.get(name, 0) + Fraction(j) ** m
                else:
                    known += val * Fraction(j) ** m
            eqs.append((c, -known))
            # D- : D- = H^-1 (B - P^T): sum_j (B[j][i] - P[j][i]) j^m - m w_i i^(m-1) = 0
            c, known = dict(target), (Fraction(-1) if (i == 0 and m == 0) else Fraction(0))
            for j in range(0, b + q + 1):
                name, val = P_entry(j, i)
                if name:
                    c[name] = c.get(name, 0) - Fraction(j) ** m
                else:
                    known -= val * Fraction(j) ** m
            eqs.append((c, -known))
    if central:
        for i in range(b):
            for j in range(i, b):
                c = {P[(i, j)]: Fraction(1)}
                c[P[(j, i)]] = c.get(P[(j, i)], 0) + Fraction(1)
                eqs.append((c, Fraction(-1) if i == j == 0 else Fraction(0)))
    for (i, j), v in free.items():
        eqs.append(({P[(i, j)]: Fraction(1)}, v))
    sol = _rref_solve(eqs, list(P.values()) + W)
    w = [sol[n] for n in W]
    cw = max(b + q, r + q + 1)   # closure rows reach b + q nodes; the kernels' q rows need
    # a window as wide as the interior stencil too (wider only for the order-2 central operator)
    dplus = [[Fraction(0)] * cw for _ in range(b)]
    dminus = [[Fraction(0)] * cw for _ in range(b)]
    for i in range(b):
        for j in range(cw):
            name, val = P_entry(i, j)
            dplus[i][j] = (sol[name] if name else val) / w[i]
            name, val = P_entry(j, i)
            bji = Fraction(-1) if (i == 0 and j == 0) else Fraction(0)
            dminus[i][j] = (bji - (sol[name] if name else val)) / w[i]
    return b, r, q, alpha, w, dplus, dminus


def _lit(x):
    return f"{x.numerator}.0/{x.denominator}.0" if x.denominator != 1 else f"{x.numerator}.0"


def render():
    out = ["// Upwind SBP dual-pair coefficients (orders 2 to 7) and the traditional central operators",
           "// (orders 2, 4, 6; OpCoef<kTraditional + order>, D- = D+) for the CUDA kernels.",
           "// Generated by paper_2011_02600_gb300/opgen.py from Table 1 of arXiv 2011.02600 and the",
           "// closure conditions stated there; do not edit by hand.",
           "#pragma once", "", "#ifndef __CUDACC__", "#define __host__", "#define __device__", "#endif", "",
           "namespace sbp {", "", "template <int ORDER> struct OpCoef;", "",
           f"constexpr int kTraditional = {TRADITIONAL};  // OpCoef<kTraditional + order>: Table 2's operator", ""]
    for order in ORDERS + tuple(TRADITIONAL + o for o in sorted(CENTRAL)):
        b, r, q, alpha, w, dp, dm = derive(order)
        cw = len(dp[0])
        out.append(f"template <> struct OpCoef<{order}> {{")
        out.append(f"  static constexpr int b = {b}, r = {r}, q = {q}, cw = {cw};")
        if order > TRADITIONAL:
            out.append(f"  // traditional operator of order {order - TRADITIONAL}: central stencil alpha_j = -alpha_-j"
                       " (Table 2), D- = D+")
        else:
            out.append(f"  // interior D+ stencil alpha_j, j = -r..q (Table 1); 0 outside")
        expr = " : ".join(f"j == {j} ? {_lit(alpha[j])}" for j in range(-r, q + 1)) + " : 0.0"
        out.append(f"  __host__ __device__ static constexpr double alpha(int j) {{ return {expr}; }}")
        out.append("  // diagonal norm weights w_0..w_{b-1} (H = h diag(w, 1, ..., 1, reversed w)); 1 inside")
        expr = " : ".join(f"i == {i} ? {_lit(x)}" for i, x in enumerate(w)) + " : 1.0"
        out.append(f"  __host__ __device__ static constexpr double w(int i) {{ return {expr}; }}")
        out.append("};")
        out.append("")
        for nm, tab in (("dp", dp), ("dm", dm)):
            out.append(f"// {'D+' if nm == 'dp' else 'D-'} closure rows 0..{b - 1}, columns 0..{cw - 1} (unit spacing)")
            rows = ",\n  ".join("{" + ", ".join(_lit(x) for x in row) + "}" for row in tab)
            out.append(f"#define SBP_{nm.upper()}{order}_ROWS \\\n  {{{rows.replace(chr(10), ' ')}}}")
        out.append("")
    out.append("}  // namespace sbp")
    out.append("")
    return "\n".join(out)


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "sbp_coeffs.h")
    os.makedirs(os.path.dirname(path), exist_ok=True)
    text = render()
    with open(path, "w") as f:
        f.write(text)
    print(path)


if __name__ == "__main__":
    main()
