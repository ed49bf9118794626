// Weights of the 1D discrete delta of a point source (host code, used by sbp_set_sources in
// api.cu): the paper gives the source term of Eq. momententor_pointsource but not its
// discretisation; the weights satisfy the discrete moment conditions up to degree m on m + 1
// consecutive nodes.
#pragma once

#include <math.h>

#include <algorithm>
#include <utility>
#include <vector>

namespace sbp {

// 1D discrete delta: m+1 consecutive nodes from floor(xi0/h) - (m-1)/2 (centred on the
// source's cell, shifted inwards at a face), moment conditions up to degree m.
inline void delta_1d(double xi0, int N, int m, int* start, double* phi) {
  const double h = 1.0 / (N - 1);
  int c = (int)floor(xi0 / h) - (m - 1) / 2;
  c = std::max(0, std::min(N - 1 - m, c));
  *start = c;
  // solve V^T phi = e0 with V[k][i] = x_i^k (Gaussian elimination, partial pivoting)
  const int n = m + 1;
  std::vector<double> A(n * (n + 1));
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < n; ++i) A[k * (n + 1) + i] = pow(((c + i) * h - xi0) / h, k);
    A[k * (n + 1) + n] = k == 0 ? 1.0 : 0.0;
  }
  for (int col = 0; col < n; ++col) {
    int p = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(A[r * (n + 1) + col]) > fabs(A[p * (n + 1) + col])) p = r;
    for (int x = 0; x <= n; ++x) std::swap(A[col * (n + 1) + x], A[p * (n + 1) + x]);
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[r * (n + 1) + col] / A[col * (n + 1) + col];
      for (int x = col; x <= n; ++x) A[r * (n + 1) + x] -= f * A[col * (n + 1) + x];
    }
  }
  for (int i = 0; i < n; ++i) phi[i] = A[i * (n + 1) + n] / A[i * (n + 1) + i];
}

}  // namespace sbp
