// Discrete adjoint of the fused stage, material gradient and receiver misfit.
//
// Forward stage k of the 2N-storage scheme: W_k = A_k W_{k-1} + dt (L U_k + f_k),
// U_{k+1} = U_k + B_k W_k with L = P~ M (M: the raw operator, penalties included).
// Its exact adjoint, run for k = 4..0:
//     Wb_k  = Wb + B_k Ub_{k+1}               (Wb holds A_{k+1} Wb_{k+1})
//     Ub_k  = Ub_{k+1} + dt L^T Wb_k
//     Wb   <- A_k Wb_k
//     g    += dt (d(L U_k)/dm)^T Wb_k          (m = rho, lambda, mu per node)
//
// L^T = M^T P~.  With the dual-pair relation H D+ + D-^T H = B (Section 4.1,
// Eq. upw_SBP) the transposes are D-^T = B H^-1 - H D+ H^-1 and
// D+^T = B H^-1 - H D- H^-1, so with y = P~ Wb_k and yh = H^-1 y (pointwise):
//     vb     = sum_xi [ -H D-_xi F_xi(yh_sigma) + (B H^-1)_xi F_xi(y_sigma) ] + (SAT^T y)_v
//     sigmab = sum_xi [ -H sym(a_xi (x) D+_xi yh_v) + (B H^-1)_xi sym(a_xi (x) y_v) ] + (SAT^T y)_sigma
// i.e. the forward operator's own rows applied to yh, plus face terms.
#include <math.h>

#include "common.cuh"
#include "launch.h"

namespace sbp {

template <int O>
__device__ __forceinline__ double node_weight(const Dims& d, int i, int j, int k) {
  return norm_weight<O>(i, d.nq) / (d.nq - 1) * norm_weight<O>(j, d.nr) / (d.nr - 1) * norm_weight<O>(k, d.ns) /
         (d.ns - 1);
}

template <typename T, int O>
__global__ void adjoint_prep_kernel(AdjArgs<T> A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const Dims d = A.d;
  if (t >= (long long)d.nq * d.nr * d.ns) return;
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
  const T ih = T(1.0 / node_weight<O>(d, i, j, k));
#pragma unroll
  for (int f = 0; f < 9; ++f) A.yhat[f * fs + n0] = y[f] * ih;
}

// Transposed penalty of one face at one node: (vb, sb) += SAT^T (y_v, y_sigma).
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

template <typename T, int O>
__global__ void __launch_bounds__(256) adjoint_stage_kernel(AdjArgs<T> A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const Dims d = A.d;
  if (t >= (long long)d.nq * d.nr * d.ns) return;
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
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const bool lo = pos[xi] == 0, hi = pos[xi] == N[xi] - 1;
    if (!(lo || hi)) continue;
    const T* __restrict__ mx = A.met + (long long)(3 * xi) * fs;
    const T a0[3] = {mx[n0], mx[fs + n0], mx[2 * fs + n0]};
    for (int side = 0; side < 2; ++side) {
      if ((side == 0 && !lo) || (side == 1 && !hi)) continue;
      const T sg = side == 0 ? -A.inv_h0[xi] : A.inv_h0[xi];
      T F[3];
      flux(a0, y + 3, F);
      vb[0] += sg * F[0];
      vb[1] += sg * F[1];
      vb[2] += sg * F[2];
      const T u[3] = {sg * y[0], sg * y[1], sg * y[2]};
      add_strain(a0, u, sb);
      add_penalty_transpose<T>(side, A.bc_kind[2 * xi + side], A.bc_gamma[2 * xi + side], A.inv_h0[xi], y, y + 3,
                               a0, irhoJ, lamJ, muJ, vb, sb);
    }
  }
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
  const double rho = A.rlmj[n0], lam = A.rlmj[fs + n0], mu = A.rlmj[2 * fs + n0], J = A.rlmj[3 * fs + n0];
  const double dt = (double)A.dt;
  const double wv = (double)rv[0] * wk[0] + (double)rv[1] * wk[1] + (double)rv[2] * wk[2];
  const double tre = (double)e[0] + e[1] + e[2];
  double g_rho = -dt * wv / (rho * rho * J);
  double g_lam = dt * tre / J * ((double)wk[3] + wk[4] + wk[5]);
  double g_mu = dt / J * (2.0 * ((double)e[0] * wk[3] + (double)e[1] * wk[4] + (double)e[2] * wk[5]) +
                          (double)e[3] * wk[6] + (double)e[4] * wk[7] + (double)e[5] * wk[8]);
  // impedances in the general penalty
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const bool lo = pos[xi] == 0, hi = pos[xi] == N[xi] - 1;
    if (!(lo || hi)) continue;
    const T* __restrict__ mx = A.met + (long long)(3 * xi) * fs;
    const T a0[3] = {mx[n0], mx[fs + n0], mx[2 * fs + n0]};
    for (int side = 0; side < 2; ++side) {
      if ((side == 0 && !lo) || (side == 1 && !hi)) continue;
      if (A.bc_kind[2 * xi + side] != 1) continue;
      const T Zp = sqrt((lamJ + T(2) * muJ) / irhoJ), Zs = sqrt(muJ / irhoJ);
      T dZp, dZs;
      penalty_impedance_derivs<T>(side, A.bc_gamma[2 * xi + side], A.inv_h0[xi], qc, qc + 3, y, y + 3, a0, Zp, Zs,
                                  dZp, dZs);
      const double zp = sqrt(rho * (lam + 2.0 * mu)), zs = sqrt(rho * mu);
      g_rho += dt * ((double)dZp * (lam + 2.0 * mu) / (2.0 * zp) + (double)dZs * mu / (2.0 * zs));
      g_lam += dt * (double)dZp * rho / (2.0 * zp);
      g_mu += dt * ((double)dZp * rho / zp + (double)dZs * rho / (2.0 * zs));
    }
  }
  A.grad[n0] += g_rho;
  A.grad[fs + n0] += g_lam;
  A.grad[2 * fs + n0] += g_mu;
}

template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T>& A, int order, cudaStream_t st) {
  const long long total = (long long)A.d.nq * A.d.nr * A.d.ns;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  switch (order) {
    case 2: adjoint_prep_kernel<T, 2><<<blocks, 256, 0, st>>>(A); break;
    case 4: adjoint_prep_kernel<T, 4><<<blocks, 256, 0, st>>>(A); break;
    case 6: adjoint_prep_kernel<T, 6><<<blocks, 256, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (order) {
    case 2: adjoint_stage_kernel<T, 2><<<blocks, 256, 0, st>>>(A); break;
    case 4: adjoint_stage_kernel<T, 4><<<blocks, 256, 0, st>>>(A); break;
    case 6: adjoint_stage_kernel<T, 6><<<blocks, 256, 0, st>>>(A); break;
  }
  return cudaGetLastError();
}

// Receivers: misfit 1/2 w (v - d)^2 accumulated per receiver component in FP64, and the
// adjoint source w (v - d) added to ubar (if given) at the receiver node.
template <typename T>
__global__ void misfit_kernel(const T* __restrict__ q, Dims d, const int32_t* __restrict__ off, int n,
                              const double* __restrict__ data, double w, double* __restrict__ acc, T* ubar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 3) return;
  const int r = t / 3, c = t % 3;
  const long long idx = (long long)c * d.fs + off[r];
  const double diff = (double)q[idx] - data[t];
  if (acc) acc[t] += 0.5 * w * diff * diff;
  if (ubar) ubar[idx] = (T)((double)ubar[idx] + w * diff);
}

template <typename T>
cudaError_t launch_misfit(const T* q, const Dims& d, const int32_t* off, int n, const double* data, double w,
                          double* acc, T* ubar, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  misfit_kernel<T><<<(n * 3 + 127) / 128, 128, 0, st>>>(q, d, off, n, data, w, acc, ubar);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint<float>(const AdjArgs<float>&, int, cudaStream_t);
template cudaError_t launch_adjoint<double>(const AdjArgs<double>&, int, cudaStream_t);
template cudaError_t launch_misfit<float>(const float*, const Dims&, const int32_t*, int, const double*, double,
                                          double*, float*, cudaStream_t);
template cudaError_t launch_misfit<double>(const double*, const Dims&, const int32_t*, int, const double*, double,
                                           double*, double*, cudaStream_t);

}  // namespace sbp
