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
#include "source_weights.h"

using namespace sbp;

template <typename T, int O>
static void rhs_all(int nq, int nr, int ns, const T* q, const T* met, const T* mat, const int* bc_kind,
                    const double* bc_gamma, T* out) {
  Dims d;
  d.nq = nq;
  d.nr = nr;
  d.ns = ns;
  d.ldq = nq;
  d.plane = nq * nr;
  d.fs = (long long)nq * nr * ns;
  const int N[3] = {nq, nr, ns};
  // the kernels' parameters as the library forms them (make_args in api.cu)
  T inv_h[3], inv_h0[3];
  for (int x = 0; x < 3; ++x) {
    inv_h[x] = (T)(N[x] - 1);
    inv_h0[x] = (T)((double)(N[x] - 1) / OpCoef<O>::w(0));
  }
  int kind[6];
  T gamma[6];
  for (int f = 0; f < 6; ++f) {
    kind[f] = bc_kind[f];
    gamma[f] = (T)bc_gamma[f];
  }
  for (int k = 0; k < ns; ++k)
    for (int j = 0; j < nr; ++j)
      for (int i = 0; i < nq; ++i) {
        const long long n0 = (long long)k * d.plane + (long long)j * nq + i;
        const int pos[3] = {i, j, k};
        T rv[3], e[6], qc[9], dq[9];
        raw_operator_at<T, O>(q, met, mat, d, n0, pos, inv_h, inv_h0, kind, gamma, rv, e, qc);
        apply_P(rv, e, mat[n0], mat[d.fs + n0], mat[2 * d.fs + n0], dq);
        for (int f = 0; f < 9; ++f) out[f * d.fs + n0] = dq[f];
      }
}

template <typename T>
static int rhs_order(int order, int nq, int nr, int ns, const T* q, const T* met, const T* mat, const int* bc_kind,
                     const double* bc_gamma, T* out) {
  switch (order) {
    case 2: rhs_all<T, 2>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case 3: rhs_all<T, 3>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case 4: rhs_all<T, 4>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case 5: rhs_all<T, 5>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case 6: rhs_all<T, 6>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case 7: rhs_all<T, 7>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case kTraditional + 2: rhs_all<T, kTraditional + 2>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case kTraditional + 4: rhs_all<T, kTraditional + 4>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    case kTraditional + 6: rhs_all<T, kTraditional + 6>(nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out); return 0;
    default: return 1;
  }
}

// FP64 (double arrays) or FP32 (float arrays: state, metrics and coefficients in FP32, as the
// library stores them for a precision-32 grid).
extern "C" int host_rhs(int order, int nq, int nr, int ns, const double* q, const double* met, const double* mat,
                        const int* bc_kind, const double* bc_gamma, double* out) {
  return rhs_order<double>(order, nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out);
}
extern "C" int host_rhs_f32(int order, int nq, int nr, int ns, const float* q, const float* met, const float* mat,
                            const int* bc_kind, const double* bc_gamma, float* out) {
  return rhs_order<float>(order, nq, nr, ns, q, met, mat, bc_kind, bc_gamma, out);
}

// Discrete energy E = 1/2 sum_nodes H J (rho |v|^2 + sigma^T S sigma) from the kernels' per-node
// energy_density (common.cuh) and norm weights, FP64, summed node by node.
template <int O>
static double energy_all(int nq, int nr, int ns, const double* q, const double* mat) {
  const long long fs = (long long)nq * nr * ns;
  double E = 0.0;
  for (int k = 0; k < ns; ++k)
    for (int j = 0; j < nr; ++j)
      for (int i = 0; i < nq; ++i) {
        const long long n0 = ((long long)k * nr + j) * nq + i;
        double v[3], s[6];
        for (int c = 0; c < 3; ++c) v[c] = q[c * fs + n0];
        for (int c = 0; c < 6; ++c) s[c] = q[(3 + c) * fs + n0];
        const double H = norm_weight<O>(i, nq) / (nq - 1) * norm_weight<O>(j, nr) / (nr - 1) * norm_weight<O>(k, ns) /
                         (ns - 1);
        E += H * energy_density<double>(v, s, mat[n0], mat[fs + n0], mat[2 * fs + n0]);
      }
  return 0.5 * E;
}

extern "C" int host_energy(int order, int nq, int nr, int ns, const double* q, const double* mat, double* out) {
  switch (order) {
    case 2: *out = energy_all<2>(nq, nr, ns, q, mat); return 0;
    case 3: *out = energy_all<3>(nq, nr, ns, q, mat); return 0;
    case 4: *out = energy_all<4>(nq, nr, ns, q, mat); return 0;
    case 5: *out = energy_all<5>(nq, nr, ns, q, mat); return 0;
    case 6: *out = energy_all<6>(nq, nr, ns, q, mat); return 0;
    case 7: *out = energy_all<7>(nq, nr, ns, q, mat); return 0;
    case kTraditional + 2: *out = energy_all<kTraditional + 2>(nq, nr, ns, q, mat); return 0;
    case kTraditional + 4: *out = energy_all<kTraditional + 4>(nq, nr, ns, q, mat); return 0;
    case kTraditional + 6: *out = energy_all<kTraditional + 6>(nq, nr, ns, q, mat); return 0;
    default: return 1;
  }
}

// J and the metric terms (metrics_at of common.cuh) at every node of a densely stored grid:
// xyz 3 fields, jmet 10 fields (J, then a[xi][eta]).  Returns the number of nodes with J <= 0.
template <int O>
static long long metrics_all(int nq, int nr, int ns, const double* xyz, double* jmet) {
  Dims d;
  d.nq = nq;
  d.nr = nr;
  d.ns = ns;
  d.ldq = nq;
  d.plane = nq * nr;
  d.fs = (long long)nq * nr * ns;
  long long bad = 0;
  for (long long t = 0; t < d.fs; ++t) bad += metrics_at<O>(xyz, jmet, d, t) ? 0 : 1;
  return bad;
}

extern "C" long long host_metrics(int order, int nq, int nr, int ns, const double* xyz, double* jmet) {
  switch (order) {
    case 2: return metrics_all<2>(nq, nr, ns, xyz, jmet);
    case 3: return metrics_all<3>(nq, nr, ns, xyz, jmet);
    case 4: return metrics_all<4>(nq, nr, ns, xyz, jmet);
    case 5: return metrics_all<5>(nq, nr, ns, xyz, jmet);
    case 6: return metrics_all<6>(nq, nr, ns, xyz, jmet);
    case 7: return metrics_all<7>(nq, nr, ns, xyz, jmet);
    default: return -1;
  }
}

// The point source's 1D discrete-delta weights as the library computes them (source_weights.h).
extern "C" int host_delta_1d(double xi0, int N, int m, int* start, double* phi) {
  if (m < 1 || m > 7 || N < m + 1) return 1;
  sbp::delta_1d(xi0, N, m, start, phi);
  return 0;
}
