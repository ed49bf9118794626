// CPU check of the tiled stage kernel's index arithmetic (paper_2011_02600_gb300/csrc/tile_map.cuh,
// compiled here as host C++) for every grid size in a range, for the upwind orders 2 to 7 and the
// traditional operators of orders 2, 4, 6 (the kernels are launched for the upwind orders 2, 4
// and 6; the others are checked ahead of their GPU runs):
//   * the tiles along q (width TX, origins on 4-node boundaries) and r (width TY) own disjoint
//     node ranges that cover the axis, and every q origin keeps the tile loads on a 16-byte
//     boundary;
//   * the per-thread q rows (fill_q_rows): every tap of every thread lies in the flux columns the
//     kernel computes and in the loaded state columns, threads that own no node carry zero
//     weights, and the row a thread applies equals row i of D- and of D+ (Table 1 inside, the
//     closure tables within b of a face, the mirrored closure at the far face);
//   * along r, every tap of every owned node's rows lies in the computed flux rows and the loaded
//     state rows of its tile;
//   * the tile launch order (swizzle_tiles) is a bijection onto the tiles;
//   * apply_row (the rows of the general, metrics and adjoint kernels) equals the dense rows, the
//     norm weights are symmetric and integrate constants exactly, and the applied operators
//     satisfy the SBP relation H D+ + D-^T H = B (Sec. 4.1, Eq. upw_SBP) to rounding;
//   * the closure-row sums along s (s_closure_sums) equal the closure rows of D- applied to
//     F_s = sigma a_s and of D+ applied to v, at both ends.
// Prints "ok" and exits 0, or lists the first failures and exits 1.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

using std::max;
using std::min;

#define __ldg(p) (*(p))   // the read-only-cache load of the kernel is a plain load on the host
#include "tile_map.cuh"

using namespace sbp;

static long failures = 0;
#define CHECK(cond, ...)                 \
  do {                                   \
    if (!(cond)) {                       \
      if (failures++ < 20) {             \
        fprintf(stderr, __VA_ARGS__);    \
        fputc('\n', stderr);             \
      }                                  \
    }                                    \
  } while (0)

// Closure tables of D+ and D- (rows 0..b-1, columns 0..cw-1, unit spacing).
template <int O> struct Closure;
template <> struct Closure<2> {
  static constexpr double P[2][4] = SBP_DP2_ROWS;
  static constexpr double M[2][4] = SBP_DM2_ROWS;
};
template <> struct Closure<4> {
  static constexpr double P[4][7] = SBP_DP4_ROWS;
  static constexpr double M[4][7] = SBP_DM4_ROWS;
};
template <> struct Closure<6> {
  static constexpr double P[6][10] = SBP_DP6_ROWS;
  static constexpr double M[6][10] = SBP_DM6_ROWS;
};
template <> struct Closure<3> {
  static constexpr double P[2][4] = SBP_DP3_ROWS;
  static constexpr double M[2][4] = SBP_DM3_ROWS;
};
template <> struct Closure<5> {
  static constexpr double P[4][7] = SBP_DP5_ROWS;
  static constexpr double M[4][7] = SBP_DM5_ROWS;
};
template <> struct Closure<7> {
  static constexpr double P[6][10] = SBP_DP7_ROWS;
  static constexpr double M[6][10] = SBP_DM7_ROWS;
};
template <> struct Closure<102> {
  static constexpr double P[1][3] = SBP_DP102_ROWS;
  static constexpr double M[1][3] = SBP_DM102_ROWS;
};
template <> struct Closure<104> {
  static constexpr double P[4][6] = SBP_DP104_ROWS;
  static constexpr double M[4][6] = SBP_DM104_ROWS;
};
template <> struct Closure<106> {
  static constexpr double P[6][9] = SBP_DP106_ROWS;
  static constexpr double M[6][9] = SBP_DM106_ROWS;
};

// Row i of D+ (plus) or D- on n nodes as a dense vector: the closure rows within b of the
// q = 0 face, at the far face D+[n-1-i][n-1-j] = -D-[i][j] and D-[n-1-i][n-1-j] = -D+[i][j],
// and inside alpha_j at offsets -r..q for D+, beta_j = -alpha_{-j} at offsets -q..r for D-.
template <int O>
std::vector<double> dense_row(int i, int n, bool plus) {
  using C = OpCoef<O>;
  std::vector<double> row(n, 0.0);
  if (i < C::b) {
    for (int c = 0; c < C::cw; ++c) row[c] = plus ? Closure<O>::P[i][c] : Closure<O>::M[i][c];
  } else if (i > n - 1 - C::b) {
    const int ii = n - 1 - i;
    for (int c = 0; c < C::cw; ++c) row[n - 1 - c] = plus ? -Closure<O>::M[ii][c] : -Closure<O>::P[ii][c];
  } else if (plus) {
    for (int j = -C::r; j <= C::q; ++j) row[i + j] = C::alpha(j);
  } else {
    for (int j = -C::q; j <= C::r; ++j) row[i + j] = -C::alpha(-j);
  }
  return row;
}

// Ownership along one axis: disjoint ranges covering [0, n), origins as required.
void check_partition(int n, int w, int align, const char* axis) {
  const int nt = (n + w - 1) / w;
  int next = 0;
  for (int t = 0; t < nt; ++t) {
    const TileAxis a = tile_axis(t, nt, n, w, align);
    CHECK(a.own0 == next, "%s n=%d tile %d: owns from %d, expected %d", axis, n, t, a.own0, next);
    CHECK(a.own1 > a.own0 && a.own1 - a.own0 <= w, "%s n=%d tile %d: owns [%d, %d)", axis, n, t, a.own0, a.own1);
    CHECK(a.origin == a.own0 && a.origin >= 0 && a.origin % align == 0, "%s n=%d tile %d: origin %d", axis, n, t,
          a.origin);
    next = a.own1;
  }
  CHECK(next == n, "%s n=%d: ownership ends at %d", axis, n, next);
}

template <typename T, int O>
void check_q_rows(int n) {
  using C = OpCoef<O>;
  constexpr int CW = C::cw, R = C::r;
  const int nt = (n + TX - 1) / TX;
  static QRows<T> Qr;
  for (int t = 0; t < nt; ++t) {
    const TileAxis a = tile_axis(t, nt, n, TX, 4);
    for (int tx = 0; tx < TX; ++tx) {
      fill_q_rows<T, O>(Qr, tx, a.origin, a.own0, a.own1, n);
      const int bm = Qr.bm[tx], bp = Qr.bp[tx];
      CHECK(bm >= HX - flux_halo<O>() && bm + CW <= HX + TX + R,
            "q n=%d O=%d tile %d tx %d: D- taps [%d, %d) outside the flux columns",
            n, O, t, tx, bm, bm + CW);
      CHECK(bp >= 0 && bp + CW <= BXH, "q n=%d O=%d tile %d tx %d: D+ taps [%d, %d) outside the state columns", n, O, t, tx,
            bp, bp + CW);
      for (int c = CW; c < kMaxCW; ++c)
        CHECK(Qr.wm[c][tx] == T(0) && Qr.wp[c][tx] == T(0), "q n=%d O=%d: weight beyond cw", n, O);
      const int i = a.origin + tx;
      const bool owned = i >= a.own0 && i < a.own1;
      if (!owned) {
        for (int c = 0; c < CW; ++c)
          CHECK(Qr.wm[c][tx] == T(0) && Qr.wp[c][tx] == T(0), "q n=%d O=%d tile %d tx %d: weight on a column not owned", n,
                O, t, tx);
        continue;
      }
      for (int pass = 0; pass < 2; ++pass) {
        const bool plus = pass == 1;
        std::vector<double> eff(n, 0.0);
        for (int c = 0; c < CW; ++c) {
          const T wgt = plus ? Qr.wp[c][tx] : Qr.wm[c][tx];
          const int node = a.origin - HX + (plus ? bp : bm) + c;   // smem column 0 is node origin - HX
          if (wgt == T(0)) continue;
          CHECK(node >= 0 && node < n, "q n=%d O=%d node %d: tap at node %d outside the grid", n, O, i, node);
          if (node >= 0 && node < n) eff[node] += (double)wgt;
        }
        const std::vector<double> want = dense_row<O>(i, n, plus);
        for (int c = 0; c < n; ++c)
          CHECK(eff[c] == (double)(T)want[c], "q n=%d O=%d node %d: %s row differs at node %d (%.17g vs %.17g)", n, O, i,
                plus ? "D+" : "D-", c, eff[c], (double)(T)want[c]);
      }
    }
  }
}

template <int O>
void check_r_taps(int n) {
  using C = OpCoef<O>;
  const int nt = (n + TY - 1) / TY;
  for (int t = 0; t < nt; ++t) {
    const TileAxis a = tile_axis(t, nt, n, TY, 1);
    for (int j = a.own0; j < a.own1; ++j)
      for (int pass = 0; pass < 2; ++pass) {
        const bool plus = pass == 1;
        const std::vector<double> row = dense_row<O>(j, n, plus);
        for (int c = 0; c < n; ++c) {
          if (row[c] == 0.0) continue;
          const int s = c - a.origin + HX;   // smem row of node c
          if (plus)
            CHECK(s >= 0 && s < BYH, "r n=%d O=%d node %d: D+ tap at node %d outside the state rows", n, O, j, c);
          else
            CHECK(s >= HX - flux_halo<O>() && s < HX + TY + C::r, "r n=%d O=%d node %d: D- tap at node %d outside the flux rows", n,
                  O, j, c);
        }
      }
  }
}

// apply_row (the rows the general, metrics and adjoint kernels apply) equals the dense rows.
template <typename T, int O>
void check_apply_row(int n) {
  for (int pos = 0; pos < n; ++pos)
    for (int pass = 0; pass < 2; ++pass) {
      const bool plus = pass == 1;
      std::vector<double> eff(n, 0.0);
      bool inside = true;
      auto fn = [&](int c, T w) {
        if (c < 0 || c >= n) inside = false;
        else eff[c] += (double)w;
      };
      if (plus) apply_row<T, O, true>(pos, n, fn);
      else apply_row<T, O, false>(pos, n, fn);
      CHECK(inside, "apply_row n=%d O=%d pos %d: tap outside the grid", n, O, pos);
      const std::vector<double> want = dense_row<O>(pos, n, plus);
      for (int c = 0; c < n; ++c)
        CHECK(eff[c] == (double)(T)want[c], "apply_row n=%d O=%d pos %d: %s row differs at %d", n, O, pos,
              plus ? "D+" : "D-", c);
    }
}

// Norm weights: symmetric, sum n - 1 (H integrates constants exactly on unit spacing), and the
// compile-time forms in T equal the rounded weight and its reciprocal.
template <int O>
void check_weights(int n) {
  double sum = 0.0;
  for (int i = 0; i < n; ++i) {
    const double w = norm_weight<O>(i, n);
    sum += w;
    CHECK(w > 0.0 && w == norm_weight<O>(n - 1 - i, n), "weights n=%d O=%d: w[%d] = %g", n, O, i, w);
    CHECK((norm_weight_t<float, O>(i, n) == (float)w && norm_weight_t<double, O>(i, n) == w),
          "weights n=%d O=%d: constant form of w[%d]", n, O, i);
    CHECK((norm_weight_inv_t<float, O>(i, n) == (float)(1.0 / w) && norm_weight_inv_t<double, O>(i, n) == 1.0 / w),
          "weights n=%d O=%d: constant form of 1/w[%d]", n, O, i);
  }
  CHECK(sum > n - 1 - 1e-12 * n && sum < n - 1 + 1e-12 * n, "weights n=%d O=%d: sum %.17g", n, O, sum);
}

// The SBP relation H D+ + D-^T H = diag(-1, 0, ..., 0, 1) (Sec. 4.1, Eq. upw_SBP) for the
// operators the kernels apply, to rounding.
template <int O>
void check_sbp(int n) {
  std::vector<double> P((size_t)n * n, 0.0), M((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    apply_row<double, O, true>(i, n, [&](int c, double w) { P[(size_t)i * n + c] += w; });
    apply_row<double, O, false>(i, n, [&](int c, double w) { M[(size_t)i * n + c] += w; });
  }
  double worst = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double v = norm_weight<O>(i, n) * P[(size_t)i * n + j] + M[(size_t)j * n + i] * norm_weight<O>(j, n);
      const double b = i == j ? (i == 0 ? -1.0 : i == n - 1 ? 1.0 : 0.0) : 0.0;
      worst = max(worst, v - b > 0 ? v - b : b - v);
    }
  CHECK(worst < 1e-13, "SBP relation n=%d O=%d: residual %g", n, O, worst);
}

// s_closure_sums on one node column: scratch row (end, r, c) = row r (or ns-1-r) of D- applied
// to F_s,c = (sigma a_s)_c along s, and of D+ applied to v_c.
template <typename T, int O>
void check_s_closure(int ns) {
  using C = OpCoef<O>;
  Dims d;
  d.nq = 1;
  d.nr = 1;
  d.ns = ns;
  d.ldq = 1;
  d.plane = 1;
  d.fs = ns;
  std::vector<T> q(9 * (size_t)ns), met(9 * (size_t)ns), scratch(2 * C::b * 6, T(-1));
  unsigned x = 12345u + ns;
  for (auto& v : q) v = T(((x = x * 1664525u + 1013904223u) >> 8) / double(1 << 24) - 0.5);
  for (auto& v : met) v = T(((x = x * 1664525u + 1013904223u) >> 8) / double(1 << 24) - 0.5);
  s_closure_sums<T, O, false>(q.data(), met.data(), d, 0, scratch.data());
  s_closure_sums<T, O, true>(q.data(), met.data(), d, 0, scratch.data());
  std::vector<double> F[3], v[3];
  for (int c = 0; c < 3; ++c) {
    F[c].assign(ns, 0.0);
    v[c].assign(ns, 0.0);
  }
  for (int k = 0; k < ns; ++k) {
    const double a0 = met[6 * ns + k], a1 = met[7 * ns + k], a2 = met[8 * ns + k];
    const double sg[6] = {q[3 * ns + k], q[4 * ns + k], q[5 * ns + k], q[6 * ns + k], q[7 * ns + k], q[8 * ns + k]};
    F[0][k] = a0 * sg[0] + a1 * sg[3] + a2 * sg[4];   // sigma a_s with sigma in Voigt order xx yy zz xy xz yz
    F[1][k] = a0 * sg[3] + a1 * sg[1] + a2 * sg[5];
    F[2][k] = a0 * sg[4] + a1 * sg[5] + a2 * sg[2];
    for (int c = 0; c < 3; ++c) v[c][k] = q[c * ns + k];
  }
  const double tol = sizeof(T) == 8 ? 1e-13 : 1e-5;
  for (int e = 0; e < 2; ++e)
    for (int r = 0; r < C::b; ++r) {
      const int plane = e ? ns - 1 - r : r;
      const std::vector<double> rm = dense_row<O>(plane, ns, false), rp = dense_row<O>(plane, ns, true);
      for (int c = 0; c < 3; ++c) {
        double wm = 0.0, wp = 0.0, scale = 0.0;
        for (int k = 0; k < ns; ++k) {
          wm += rm[k] * F[c][k];
          wp += rp[k] * v[c][k];
          scale += std::fabs(rm[k]) + std::fabs(rp[k]);
        }
        const double gm = scratch[(e * C::b + r) * 6 + c], gp = scratch[(e * C::b + r) * 6 + 3 + c];
        CHECK(std::fabs(gm - wm) <= tol * scale && std::fabs(gp - wp) <= tol * scale,
              "s closure ns=%d O=%d end %d row %d c %d: (%g, %g) vs (%g, %g)", ns, O, e, r, c, gm, gp, wm, wp);
      }
    }
}

void check_swizzle(int nbx, int nby) {
  std::vector<char> seen((size_t)nbx * nby, 0);
  for (int lin = 0; lin < nbx * nby; ++lin) {
    int bx = -1, by = -1;
    swizzle_tiles(lin, nbx, nby, bx, by);
    const bool in = bx >= 0 && bx < nbx && by >= 0 && by < nby;
    CHECK(in, "swizzle %d x %d: launch %d maps to (%d, %d)", nbx, nby, lin, bx, by);
    if (in) {
      CHECK(!seen[(size_t)by * nbx + bx], "swizzle %d x %d: tile (%d, %d) launched twice", nbx, nby, bx, by);
      seen[(size_t)by * nbx + bx] = 1;
    }
  }
}

template <int O>
void check_order(const std::vector<int>& sizes) {
  const int nmin = 2 * OpCoef<O>::b + max(OpCoef<O>::r, OpCoef<O>::q);
  for (int n : sizes) {
    if (n < nmin) continue;
    check_partition(n, TX, 4, "q");
    check_partition(n, TY, 1, "r");
    check_q_rows<double, O>(n);
    check_q_rows<float, O>(n);
    check_r_taps<O>(n);
    check_apply_row<double, O>(n);
    check_apply_row<float, O>(n);
    check_weights<O>(n);
    check_s_closure<double, O>(n);
    check_s_closure<float, O>(n);
    if (n <= 64) check_sbp<O>(n);
  }
}

int main() {
  std::vector<int> sizes;
  for (int n = 1; n <= 400; ++n) sizes.push_back(n);
  for (int n : {511, 512, 513, 1023, 1024, 1025, 1026, 1029, 2049, 4097}) sizes.push_back(n);
  check_order<2>(sizes);
  check_order<3>(sizes);
  check_order<4>(sizes);
  check_order<5>(sizes);
  check_order<6>(sizes);
  check_order<7>(sizes);
  check_order<kTraditional + 2>(sizes);
  check_order<kTraditional + 4>(sizes);
  check_order<kTraditional + 6>(sizes);
  for (int nbx = 1; nbx <= 70; ++nbx)
    for (int nby = 1; nby <= 140; ++nby) check_swizzle(nbx, nby);
  if (failures) {
    fprintf(stderr, "%ld failures\n", failures);
    return 1;
  }
  printf("ok\n");
  return 0;
}
