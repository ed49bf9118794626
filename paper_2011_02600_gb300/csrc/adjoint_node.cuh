// Per-node bodies of the general adjoint kernels (kernels_adjoint.cu, where the scheme is
// written out): the prep pass (Wb_k = Wb + B_k Ub_{k+1}, yhat = H^-1 P~ Wb_k) and the stage pass
// (L^T on yhat with the face terms, the Runge-Kutta updates of Ub and Wb, and the material
// gradient) at node t of the [s][r][q] enumeration.  Device code of those kernels; without
// nvcc the same source compiles as host C++, so that the adjoint can be checked on a CPU.
#pragma once

#include "adjoint_args.h"
#include "adjoint_terms.cuh"
#include "common.cuh"

namespace sbp {

// Gradient accumulation: the members of a batch add to the same node, so the device adds
// atomically (the host build, one thread, adds directly).
__device__ __forceinline__ void grad_add(double* p, double v) {
#ifdef __CUDA_ARCH__
  atomicAdd(p, v);
#else
  *p += v;
#endif
}

// The buffers of batch member b (every 9-field buffer advanced by b member strides; the
// gradient, the coefficients and rho, lambda, mu, J are shared by the members).
template <typename T>
__device__ __forceinline__ AdjArgs<T> adjoint_member(AdjArgs<T> A, int b) {
  const long long o = (long long)b * A.bstride;
  if (A.ubar_next) A.ubar_next += o;
  if (A.ubar_out) A.ubar_out += o;
  if (A.wbar_in) A.wbar_in += o;
  if (A.wbar) A.wbar += o;
  if (A.yhat) A.yhat += o;
  if (A.u) A.u += o;
  return A;
}

template <typename T, int O>
__device__ __forceinline__ void adjoint_prep_at(const AdjArgs<T>& A, long long t) {
  const Dims d = A.d;
  const int i = (int)(t % d.nq);
  const int j = (int)((t / d.nq) % d.nr);
  const int k = (int)(t / ((long long)d.nq * d.nr));
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const long long fs = d.fs;
  T w[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) {
    w[f] = A.wbar_in[f * fs + n0];
    if (A.ubar_next) w[f] += A.rk_b * A.ubar_next[f * fs + n0];
    if (A.wbar) A.wbar[f * fs + n0] = w[f];
  }
  T y[9];
  apply_P(w, w + 3, A.mat[n0], A.mat[fs + n0], A.mat[2 * fs + n0], y);
  // 1/H = (N_q - 1)(N_r - 1)(N_s - 1) / (w_i w_j w_k), without a division
  const T ih = norm_weight_inv_t<T, O>(i, d.nq) * A.inv_h[0] * norm_weight_inv_t<T, O>(j, d.nr) * A.inv_h[1] *
               norm_weight_inv_t<T, O>(k, d.ns) * A.inv_h[2];
#pragma unroll
  for (int f = 0; f < 9; ++f) A.yhat[f * fs + n0] = y[f] * ih;
}

// Transposed operator, stage updates and gradient at one node.
template <typename T, int O>
__device__ __forceinline__ void adjoint_stage_at(const AdjArgs<T>& A, long long t) {
  const Dims d = A.d;
  const int i = (int)(t % d.nq);
  const int j = (int)((t / d.nq) % d.nr);
  const int k = (int)(t / ((long long)d.nq * d.nr));
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const long long fs = d.fs;
  const int pos[3] = {i, j, k};
  const int N[3] = {d.nq, d.nr, d.ns};
  const long long stride[3] = {1, d.ldq, d.plane};
  const T H = T(node_weight<O>(d, i, j, k));
  const T* __restrict__ yh = A.yhat;

  T vb[3] = {T(0), T(0), T(0)};
  T sb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  // -H (forward rows applied to yh)
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const T* __restrict__ mx = A.met + (long long)(3 * xi) * fs;
    T fsum[3] = {T(0), T(0), T(0)};
    apply_row<T, O, false>(pos[xi], N[xi], [&](int c, T w) {
      const long long nb = n0 + (long long)(c - pos[xi]) * stride[xi];
      const T a[3] = {mx[nb], mx[fs + nb], mx[2 * fs + nb]};
      T s[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) s[m] = yh[(3 + m) * fs + nb];
      T F[3];
      flux(a, s, F);
      fsum[0] += w * F[0];
      fsum[1] += w * F[1];
      fsum[2] += w * F[2];
    });
    const T sc = -H * A.inv_h[xi];
    vb[0] += sc * fsum[0];
    vb[1] += sc * fsum[1];
    vb[2] += sc * fsum[2];
    T dv[3] = {T(0), T(0), T(0)};
    apply_row<T, O, true>(pos[xi], N[xi], [&](int c, T w) {
      const long long nb = n0 + (long long)(c - pos[xi]) * stride[xi];
      dv[0] += w * yh[nb];
      dv[1] += w * yh[fs + nb];
      dv[2] += w * yh[2 * fs + nb];
    });
    dv[0] *= sc;
    dv[1] *= sc;
    dv[2] *= sc;
    const T a0[3] = {mx[n0], mx[fs + n0], mx[2 * fs + n0]};
    add_strain(a0, dv, sb);
  }
  // face terms: (B H^-1) parts of the transposes, and the transposed penalties
  T y[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) y[f] = H * yh[f * fs + n0];
  const T irhoJ = A.mat[n0], lamJ = A.mat[fs + n0], muJ = A.mat[2 * fs + n0];
  const bool face = i == 0 || i == d.nq - 1 || j == 0 || j == d.nr - 1 || k == 0 || k == d.ns - 1;
  T a[3][3];
#pragma unroll
  for (int xi = 0; xi < 3; ++xi)
#pragma unroll
    for (int c = 0; c < 3; ++c) a[xi][c] = face ? A.met[(3 * xi + c) * fs + n0] : T(0);
  if (face) adjoint_face_terms(pos, N, a, y, irhoJ, lamJ, muJ, A.bc_kind, A.bc_gamma, A.inv_h0, vb, sb);
  const T m9[9] = {vb[0], vb[1], vb[2], sb[0], sb[1], sb[2], sb[3], sb[4], sb[5]};
  if (A.mode == 0) {
#pragma unroll
    for (int f = 0; f < 9; ++f) A.ubar_out[f * fs + n0] = m9[f];
    return;
  }
  T wk[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) wk[f] = A.wbar[f * fs + n0];
#pragma unroll
  for (int f = 0; f < 9; ++f) {
    const T un = A.ubar_next ? A.ubar_next[f * fs + n0] : T(0);
    A.ubar_out[f * fs + n0] = un + A.dt * m9[f];
    A.wbar[f * fs + n0] = A.rk_a * wk[f];
  }
  if (!A.grad || !A.u) return;
  // material gradient: dt Wb_k . d(P~ M U_k)/dm at this node
  T rv[3], e[6], qc[9];
  raw_operator_at<T, O>(A.u, A.met, A.mat, d, n0, pos, A.inv_h, A.inv_h0, A.bc_kind, A.bc_gamma, rv, e, qc);
  const double rho = A.rlmj[n0], J = A.rlmj[3 * fs + n0];
  double g[3];
  gradient_terms(rv, e, qc, wk, y, pos, N, a, irhoJ, lamJ, muJ, rho, J, A.bc_kind, A.bc_gamma, A.inv_h0,
                 (double)A.dt, g);
  const double g_rho = g[0], g_lam = g[1], g_mu = g[2];
  grad_add(A.grad + n0, g_rho);
  grad_add(A.grad + fs + n0, g_lam);
  grad_add(A.grad + 2 * fs + n0, g_mu);
}

}  // namespace sbp
