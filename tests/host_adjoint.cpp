// The general adjoint kernels' per-node bodies (adjoint_prep_at and adjoint_stage_at of
// paper_2011_02600_gb300/csrc/adjoint_node.cuh) compiled as host C++ and run over every node of
// a grid stored densely (row pitch nq, field stride nq nr ns), with the arguments set up the
// way the library sets them (adjoint_impl and make_args in api.cu).  Built by
// tests/test_host_adjoint.py.
#include <algorithm>
#include <cmath>

using std::max;
using std::min;
using std::sqrt;

#include "adjoint_node.cuh"

using namespace sbp;

template <int O>
static void run(AdjArgs<double>& A) {
  const long long total = (long long)A.d.nq * A.d.nr * A.d.ns;
  for (long long t = 0; t < total; ++t) adjoint_prep_at<double, O>(A, t);
  for (long long t = 0; t < total; ++t) adjoint_stage_at<double, O>(A, t);
}

static AdjArgs<double> args(int order, int nq, int nr, int ns, const double* met, const double* mat,
                            const int* bc_kind, const double* bc_gamma) {
  AdjArgs<double> A = {};
  A.d.nq = nq;
  A.d.nr = nr;
  A.d.ns = ns;
  A.d.ldq = nq;
  A.d.plane = nq * nr;
  A.d.fs = (long long)nq * nr * ns;
  A.met = met;
  A.mat = mat;
  const int N[3] = {nq, nr, ns};
  const double w0 = order == 2 ? OpCoef<2>::w(0) : order == 3 ? OpCoef<3>::w(0) : order == 4 ? OpCoef<4>::w(0)
                    : order == 5 ? OpCoef<5>::w(0) : order == 6 ? OpCoef<6>::w(0) : order == 7 ? OpCoef<7>::w(0)
                    : order == kTraditional + 2 ? OpCoef<kTraditional + 2>::w(0)
                    : order == kTraditional + 4 ? OpCoef<kTraditional + 4>::w(0) : OpCoef<kTraditional + 6>::w(0);
  for (int x = 0; x < 3; ++x) {
    A.inv_h[x] = N[x] - 1;
    A.inv_h0[x] = (N[x] - 1) / w0;
  }
  for (int f = 0; f < 6; ++f) {
    A.bc_kind[f] = bc_kind[f];
    A.bc_gamma[f] = bc_gamma[f];
  }
  return A;
}

static int dispatch(int order, AdjArgs<double>& A) {
  switch (order) {
    case 2: run<2>(A); return 0;
    case 3: run<3>(A); return 0;
    case 4: run<4>(A); return 0;
    case 5: run<5>(A); return 0;
    case 6: run<6>(A); return 0;
    case 7: run<7>(A); return 0;
    case kTraditional + 2: run<kTraditional + 2>(A); return 0;
    case kTraditional + 4: run<kTraditional + 4>(A); return 0;
    case kTraditional + 6: run<kTraditional + 6>(A); return 0;
    default: return 1;
  }
}

// out = L^T w (9 fields); scratch: 9 fields.
extern "C" int host_rhs_adjoint(int order, int nq, int nr, int ns, const double* w, const double* met,
                                const double* mat, const int* bc_kind, const double* bc_gamma, double* scratch,
                                double* out) {
  AdjArgs<double> A = args(order, nq, nr, ns, met, mat, bc_kind, bc_gamma);
  A.mode = 0;
  A.ubar_next = nullptr;
  A.ubar_out = out;
  A.wbar_in = w;
  A.wbar = nullptr;
  A.yhat = scratch;
  return dispatch(order, A);
}

// One adjoint stage with coefficients rk_a, rk_b and step dt: ubar, wbar updated in place,
// grad (3 FP64 fields) accumulated from the stage state u and rlmj = rho, lambda, mu, J.
extern "C" int host_adjoint_stage(int order, int nq, int nr, int ns, double rk_a, double rk_b, double dt,
                                  const double* u, double* ubar, double* wbar, double* scratch, const double* met,
                                  const double* mat, const double* rlmj, const int* bc_kind, const double* bc_gamma,
                                  double* grad) {
  AdjArgs<double> A = args(order, nq, nr, ns, met, mat, bc_kind, bc_gamma);
  A.mode = 1;
  A.ubar_next = ubar;
  A.ubar_out = ubar;
  A.wbar_in = wbar;
  A.wbar = wbar;
  A.yhat = scratch;
  A.u = u;
  A.rlmj = rlmj;
  A.grad = grad;
  A.rk_a = rk_a;
  A.rk_b = rk_b;
  A.dt = dt;
  return dispatch(order, A);
}
