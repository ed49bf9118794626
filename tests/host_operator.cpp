// The kernels' per-node operator (raw_operator_at and apply_P of
// paper_2011_02600_gb300/csrc/common.cuh: rows of D+ and D-, flux and strain forms, face
// penalties, P~) compiled as host C++, evaluated at every node of a grid stored densely
// (row pitch nq, field stride nq nr ns).  Built by tests/test_host_operator.py.
#include <algorithm>
#include <cmath>

using std::max;
using std::min;
using std::sqrt;

#include "common.cuh"

using namespace sbp;

template <int O>
static void rhs_all(int nq, int nr, int ns, const double* q, const double* met, const double* mat,
                    const int* bc_kind, const double* bc_gamma, double* out) {
  Dims d;
  d.nq = nq;
  d.nr = nr;
  d.ns = ns;
  d.ldq = nq;
  d.plane = nq * nr;
  d.fs = (long long)nq * nr * ns;
  const int N[3] = {nq, nr, ns};
  double inv_h[3], inv_h0[3];
  for (int x = 0; x < 3; ++x) {
    inv_h[x] = N[x] - 1;
    inv_h0[x] = (N[x] - 1) / OpCoef<O>::w(0);
  }
  int kind[6];
  double gamma[6];
  for (int f = 0; f < 6; ++f) {
    kind[f] = bc_kind[f];
    gamma[f] = bc_gamma[f];
  }
  for (int k = 0; k < ns; ++k)
    for (int j = 0; j < nr; ++j)
      for (int i = 0; i < nq; ++i) {
        const long long n0 = (long long)k * d.plane + (long long)j * nq + i;
        const int pos[3] = {i, j, k};
        double rv[3], e[6], qc[9], dq[9];
        raw_operator_at<double, O>(q, met, mat, d, n0, pos, inv_h, inv_h0, kind, gamma, rv, e, qc);
        apply_P(rv, e, mat[n0], mat[d.fs + n0], mat[2 * d.fs + n0], dq);
        for (int f = 0; f < 9; ++f) out[f * d.fs + n0] = dq[f];
      }
}

extern "C" int host_rhs(int order, int nq, int nr, int ns, const double* q, const double* met, const double* mat,
                        const int* bc_kind, const double* bc_gamma, double* out) {
  switch (order) {
    case 2: rhs_all<2>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case 4: rhs_all<4>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case 6: rhs_all<6>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    default: return 1;
  }
}
