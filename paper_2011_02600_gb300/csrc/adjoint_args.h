// Arguments of the general adjoint kernels (kernels_adjoint.cu, adjoint_node.cuh), kept apart
// from the launchers so that host C++ can include them without the TMA intrinsics.
#pragma once

#include "common.cuh"

namespace sbp {

template <typename T>
struct AdjArgs {
  const T* ubar_next;  // Ub_{k+1} (may be null: zero)
  T* ubar_out;         // Ub_k (mode 1) or L^T w (mode 0); may alias ubar_next
  const T* wbar_in;    // Wb before adding B_k Ub_{k+1} (mode 1), or w (mode 0)
  T* wbar;             // mode 1: Wb_k written by the prep pass, A_k Wb_k written by the stage pass
  T* yhat;             // scratch: H^-1 P~ Wb_k (9 fields)
  const T* u;          // forward stage state U_k (mode 1 with gradient)
  const T* met;
  const T* mat;
  const double* rlmj;  // rho, lambda, mu, J (FP64, 4 fields), for the gradient
  double* grad;        // d/d(rho, lambda, mu) accumulators (FP64, 3 fields), may be null
  Dims d;
  T rk_a, rk_b, dt;
  int mode;            // 0: out = L^T w; 1: adjoint stage
  int nb;              // independent states (a batch): every 9-field buffer holds nb members
  long long bstride;   // elements between consecutive members (9 fields)
  int bc_kind[6];
  T bc_gamma[6];
  T inv_h[3];
  T inv_h0[3];
};

}  // namespace sbp
