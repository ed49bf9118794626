// Per-node pieces of the discrete adjoint shared by the general adjoint kernel and the
// tiled kernel's adjoint passes: the node weight H, the face terms of L^T (the B H^-1
// parts of the transposed D-/D+ and the transposed penalties) and the material-gradient
// contraction.  See kernels_adjoint.cu for the scheme.
#pragma once

#include "common.cuh"

namespace sbp {

template <int O>
__device__ __forceinline__ double node_weight(const Dims& d, int i, int j, int k) {
  return norm_weight<O>(i, d.nq) / (d.nq - 1) * norm_weight<O>(j, d.nr) / (d.nr - 1) * norm_weight<O>(k, d.ns) /
         (d.ns - 1);
}

template <typename T>
__device__ __forceinline__ void add_penalty_transpose(int side, int kind, T gamma, T inv_h0, const T yv[3],
                                                      const T ys[6], const T a[3], T irhoJ, T lamJ, T muJ,
                                                      T vb[3], T sb[6]) {
  if (kind == 0) {
    // forward: rv += sg sigma a  ->  sb += sg sym(a (x) y_v)
    const T sg = side == 0 ? inv_h0 : -inv_h0;
    const T u[3] = {sg * yv[0], sg * yv[1], sg * yv[2]};
    add_strain(a, u, sb);
    return;
  }
  const T an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const T n[3] = {a[0] / an, a[1] / an, a[2] / an};
  const T Zp = sqrt((lamJ + T(2) * muJ) / irhoJ);
  const T Zs = sqrt(muJ / irhoJ);
  const T f = an * inv_h0;
  const T fsg = side == 0 ? f : -f;
  const T cv = T(0.5) * (T(1) - gamma);
  const T cT = T(0.5) * (T(1) + gamma) * (side == 0 ? T(-1) : T(1));
  T w[3];
  flux(n, ys, w);  // traction of y_sigma on the face
  const T un = yv[0] * n[0] + yv[1] * n[1] + yv[2] * n[2];
  const T wn = w[0] * n[0] + w[1] * n[1] + w[2] * n[2];
  const T an_ = -f * un + fsg * wn / Zp;
  T at[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) at[c] = -f * (yv[c] - un * n[c]) + fsg * (w[c] - wn * n[c]) / Zs;
#pragma unroll
  for (int c = 0; c < 3; ++c) vb[c] += cv * (Zp * an_ * n[c] + Zs * at[c]);
  const T beta[3] = {cT * (an_ * n[0] + at[0]), cT * (an_ * n[1] + at[1]), cT * (an_ * n[2] + at[2])};
  add_strain(n, beta, sb);
}

// d/dZp and d/dZs of y . SAT(U) for the general penalty (U = (v, sigma) at the node).
template <typename T>
__device__ __forceinline__ void penalty_impedance_derivs(int side, T gamma, T inv_h0, const T v[3], const T s[6],
                                                         const T yv[3], const T ys[6], const T a[3], T Zp, T Zs,
                                                         T& dZp, T& dZs) {
  const T an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const T n[3] = {a[0] / an, a[1] / an, a[2] / an};
  const T f = an * inv_h0;
  const T fsg = side == 0 ? f : -f;
  const T cv = T(0.5) * (T(1) - gamma);
  const T cT = T(0.5) * (T(1) + gamma) * (side == 0 ? T(-1) : T(1));
  T Tr[3], w[3];
  flux(n, s, Tr);
  flux(n, ys, w);
  const T vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  const T Tn = Tr[0] * n[0] + Tr[1] * n[1] + Tr[2] * n[2];
  const T un = yv[0] * n[0] + yv[1] * n[1] + yv[2] * n[2];
  const T wn = w[0] * n[0] + w[1] * n[1] + w[2] * n[2];
  T vtut = T(0), Ttwt = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    vtut += (v[c] - vn * n[c]) * (yv[c] - un * n[c]);
    Ttwt += (Tr[c] - Tn * n[c]) * (w[c] - wn * n[c]);
  }
  dZp = -f * cv * vn * un - fsg * cT * Tn * wn / (Zp * Zp);
  dZs = -f * cv * vtut - fsg * cT * Ttwt / (Zs * Zs);
}

// Face terms of L^T at one node: for each face the node lies on, (B H^-1)_xi applied to
// the flux and strain rows of y = P~ Wb (y at the node), and the transposed penalty.
template <typename T>
__device__ __forceinline__ void adjoint_face_terms(const int pos[3], const int N[3], const T a[3][3], const T y[9],
                                                   T irhoJ, T lamJ, T muJ, const int bc_kind[6], const T bc_gamma[6],
                                                   const T inv_h0[3], T vb[3], T sb[6]) {
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const bool lo = pos[xi] == 0, hi = pos[xi] == N[xi] - 1;
    if (!(lo || hi)) continue;
    for (int side = 0; side < 2; ++side) {
      if ((side == 0 && !lo) || (side == 1 && !hi)) continue;
      const T sg = side == 0 ? -inv_h0[xi] : inv_h0[xi];
      T F[3];
      flux(a[xi], y + 3, F);
      vb[0] += sg * F[0];
      vb[1] += sg * F[1];
      vb[2] += sg * F[2];
      const T u[3] = {sg * y[0], sg * y[1], sg * y[2]};
      add_strain(a[xi], u, sb);
      add_penalty_transpose<T>(side, bc_kind[2 * xi + side], bc_gamma[2 * xi + side], inv_h0[xi], y, y + 3, a[xi],
                               irhoJ, lamJ, muJ, vb, sb);
    }
  }
}

// Material gradient at one node, dt Wb_k . d(P~ M U_k)/d(rho, lambda, mu), from the raw
// operator (rv, e) of U_k (penalties included), U_k at the node (qc), Wb_k at the node
// (wk), y = P~ Wb_k at the node (read at faces only), rho and J (FP64) and the stored
// r = 1/(rho J), lambda/J, mu/J.  The three contractions are formed in the state's
// precision and scaled in FP64 by factors that need no division, 1/(rho^2 J) = r (r J) and
// 1/J = r rho, so that their tiny magnitudes cannot underflow.  At faces with the
// characteristic penalty the impedances Z_p = sqrt(rho (lambda + 2 mu)) and
// Z_s = sqrt(rho mu) add their derivatives, in the state's precision through
// dZp/drho = Zp/(2 rho), dZp/dlambda = rho/(2 Zp), dZp/dmu = rho/Zp, dZs/drho = Zs/(2 rho),
// dZs/dmu = rho/(2 Zs).
template <typename T>
__device__ __forceinline__ void gradient_terms(const T rv[3], const T e[6], const T qc[9], const T wk[9],
                                               const T y[9], const int pos[3], const int N[3], const T a[3][3],
                                               T irhoJ, T lamJ, T muJ, double rho, double J, const int bc_kind[6],
                                               const T bc_gamma[6], const T inv_h0[3], double dt, double g[3]) {
  const T wv = rv[0] * wk[0] + rv[1] * wk[1] + rv[2] * wk[2];
  const T tl = (e[0] + e[1] + e[2]) * (wk[3] + wk[4] + wk[5]);
  const T tm = T(2) * (e[0] * wk[3] + e[1] * wk[4] + e[2] * wk[5]) + e[3] * wk[6] + e[4] * wk[7] + e[5] * wk[8];
  const double r = (double)irhoJ;
  const double ir2J = r * (r * J), iJ = r * rho;
  g[0] = -dt * (double)wv * ir2J;
  g[1] = dt * (double)tl * iJ;
  g[2] = dt * (double)tm * iJ;
  const bool face = pos[0] == 0 || pos[0] == N[0] - 1 || pos[1] == 0 || pos[1] == N[1] - 1 || pos[2] == 0 ||
                    pos[2] == N[2] - 1;
  if (!face) return;
  const T Zp = sqrt((lamJ + T(2) * muJ) / irhoJ), Zs = sqrt(muJ / irhoJ);
  const T rT = T(rho), iZp = T(1) / Zp, iZs = T(1) / Zs, i2r = T(0.5) / rT;
  T d_rho = T(0), d_lam = T(0), d_mu = T(0);
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const bool lo = pos[xi] == 0, hi = pos[xi] == N[xi] - 1;
    if (!(lo || hi)) continue;
    for (int side = 0; side < 2; ++side) {
      if ((side == 0 && !lo) || (side == 1 && !hi)) continue;
      if (bc_kind[2 * xi + side] != 1) continue;
      T dZp, dZs;
      penalty_impedance_derivs<T>(side, bc_gamma[2 * xi + side], inv_h0[xi], qc, qc + 3, y, y + 3, a[xi], Zp, Zs,
                                  dZp, dZs);
      d_rho += (dZp * Zp + dZs * Zs) * i2r;
      d_lam += dZp * rT * T(0.5) * iZp;
      d_mu += dZp * rT * iZp + dZs * rT * T(0.5) * iZs;
    }
  }
  g[0] += dt * (double)d_rho;
  g[1] += dt * (double)d_lam;
  g[2] += dt * (double)d_mu;
}

}  // namespace sbp
