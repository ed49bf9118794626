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

#include "adjoint_terms.cuh"
#include "common.cuh"
#include "launch.h"

namespace sbp {

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
  // 1/H = (N_q - 1)(N_r - 1)(N_s - 1) / (w_i w_j w_k), without a division
  const T ih = norm_weight_inv_t<T, O>(i, d.nq) * A.inv_h[0] * norm_weight_inv_t<T, O>(j, d.nr) * A.inv_h[1] *
               norm_weight_inv_t<T, O>(k, d.ns) * A.inv_h[2];
#pragma unroll
  for (int f = 0; f < 9; ++f) A.yhat[f * fs + n0] = y[f] * ih;
}

// Transposed penalty of one face at one node: (vb, sb) += SAT^T (y_v, y_sigma).
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
  A.grad[n0] += g_rho;
  A.grad[fs + n0] += g_lam;
  A.grad[2 * fs + n0] += g_mu;
}

template <typename T>
cudaError_t launch_adjoint_prep(const AdjArgs<T>& A, int order, cudaStream_t st) {
  const long long total = (long long)A.d.nq * A.d.nr * A.d.ns;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  switch (order) {
    case 2: adjoint_prep_kernel<T, 2><<<blocks, 256, 0, st>>>(A); break;
    case 4: adjoint_prep_kernel<T, 4><<<blocks, 256, 0, st>>>(A); break;
    case 6: adjoint_prep_kernel<T, 6><<<blocks, 256, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T>& A, int order, cudaStream_t st) {
  cudaError_t e = launch_adjoint_prep<T>(A, order, st);
  if (e != cudaSuccess) return e;
  const long long total = (long long)A.d.nq * A.d.nr * A.d.ns;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  switch (order) {
    case 2: adjoint_stage_kernel<T, 2><<<blocks, 256, 0, st>>>(A); break;
    case 4: adjoint_stage_kernel<T, 4><<<blocks, 256, 0, st>>>(A); break;
    case 6: adjoint_stage_kernel<T, 6><<<blocks, 256, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Receivers: misfit 1/2 w (v - d)^2 accumulated per receiver component in FP64, and the
// adjoint source w (v - d) added to ubar (if given) at the receiver node.  The add is atomic:
// receivers that share a node each contribute their own source.
template <typename T>
__global__ void misfit_kernel(const T* __restrict__ q, Dims d, const int32_t* __restrict__ off, int n,
                              const double* __restrict__ data, double w, double* __restrict__ acc, T* ubar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 3) return;
  const int r = t / 3, c = t % 3;
  const long long idx = (long long)c * d.fs + off[r];
  const double diff = (double)q[idx] - data[t];
  if (acc) acc[t] += 0.5 * w * diff * diff;
  if (ubar) atomicAdd(&ubar[idx], (T)(w * diff));
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
template cudaError_t launch_adjoint_prep<float>(const AdjArgs<float>&, int, cudaStream_t);
template cudaError_t launch_adjoint_prep<double>(const AdjArgs<double>&, int, cudaStream_t);
template cudaError_t launch_misfit<float>(const float*, const Dims&, const int32_t*, int, const double*, double,
                                          double*, float*, cudaStream_t);
template cudaError_t launch_misfit<double>(const double*, const Dims&, const int32_t*, int, const double*, double,
                                           double*, double*, cudaStream_t);

}  // namespace sbp
