// General stage kernel: one thread per node of a list of boxes; every row of
// D+ and D- (interior stencil or closure), the penalties of every face the
// node lies on, and the fused Runge-Kutta stage.  It serves the boundary
// slabs (closure rows, edges, corners, penalties) and any grid too small for
// the tiled interior kernel.
#include "common.cuh"
#include "launch.h"

namespace sbp {

template <typename T, int O>
__global__ void __launch_bounds__(256) stage_general_kernel(StageArgs<T> A, BoxList L) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.off[L.n]) return;
  int bi = 0;
  while (bi < L.n - 1 && t >= L.off[bi + 1]) ++bi;
  const Box B = L.b[bi];
  const long long loc = t - L.off[bi];
  const int ni = B.i1 - B.i0, nj = B.j1 - B.j0;
  const int i = B.i0 + (int)(loc % ni);
  const long long rest = loc / ni;
  const int j = B.j0 + (int)(rest % nj);
  const int k = B.k0 + (int)(rest / nj);

  const Dims d = A.d;
  const long long fs = d.fs;
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const int pos[3] = {i, j, k};
  const int N[3] = {d.nq, d.nr, d.ns};
  const long long stride[3] = {1, d.ldq, d.plane};

  T rv[3] = {T(0), T(0), T(0)};
  T e[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const T* __restrict__ met = A.met + (long long)(3 * xi) * fs;
    // D- on the conservative flux F_xi = sigma a_xi
    T f[3] = {T(0), T(0), T(0)};
    apply_row<T, O, false>(pos[xi], N[xi], [&](int c, T w) {
      const long long nb = n0 + (long long)(c - pos[xi]) * stride[xi];
      const T a[3] = {met[nb], met[fs + nb], met[2 * fs + nb]};
      T s[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) s[m] = A.q[(3 + m) * fs + nb];
      T F[3];
      flux(a, s, F);
      f[0] += w * F[0];
      f[1] += w * F[1];
      f[2] += w * F[2];
    });
    rv[0] += A.inv_h[xi] * f[0];
    rv[1] += A.inv_h[xi] * f[1];
    rv[2] += A.inv_h[xi] * f[2];
    // D+ on the velocity, then the non-conservative product B_xi
    T dv[3] = {T(0), T(0), T(0)};
    apply_row<T, O, true>(pos[xi], N[xi], [&](int c, T w) {
      const long long nb = n0 + (long long)(c - pos[xi]) * stride[xi];
      dv[0] += w * A.q[nb];
      dv[1] += w * A.q[fs + nb];
      dv[2] += w * A.q[2 * fs + nb];
    });
    dv[0] *= A.inv_h[xi];
    dv[1] *= A.inv_h[xi];
    dv[2] *= A.inv_h[xi];
    const T a0[3] = {met[n0], met[fs + n0], met[2 * fs + n0]};
    add_strain(a0, dv, e);
  }

  T qc[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) qc[f] = A.q[f * fs + n0];
  const T irhoJ = A.mat[n0], lamJ = A.mat[fs + n0], muJ = A.mat[2 * fs + n0];
#pragma unroll
  for (int xi = 0; xi < 3; ++xi) {
    const bool lo = pos[xi] == 0, hi = pos[xi] == N[xi] - 1;
    if (!(lo || hi)) continue;
    const T* __restrict__ met = A.met + (long long)(3 * xi) * fs;
    const T a0[3] = {met[n0], met[fs + n0], met[2 * fs + n0]};
    if (lo)
      add_penalty<T>(0, A.bc_kind[2 * xi], A.bc_gamma[2 * xi], A.inv_h0[xi], qc, qc + 3, a0, irhoJ,
                     lamJ, muJ, rv, e);
    if (hi)
      add_penalty<T>(1, A.bc_kind[2 * xi + 1], A.bc_gamma[2 * xi + 1], A.inv_h0[xi], qc, qc + 3, a0,
                     irhoJ, lamJ, muJ, rv, e);
  }
  T dd[9];
  apply_P(rv, e, irhoJ, lamJ, muJ, dd);
  stage_epilogue(A, n0, dd, qc);
}

template <typename T>
cudaError_t launch_stage_general(const StageArgs<T>& A, int order, const BoxList& L, cudaStream_t st) {
  const long long total = L.off[L.n];
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = (total + threads - 1) / threads;
  switch (order) {
    case 2: stage_general_kernel<T, 2><<<(unsigned)blocks, threads, 0, st>>>(A, L); break;
    case 4: stage_general_kernel<T, 4><<<(unsigned)blocks, threads, 0, st>>>(A, L); break;
    case 6: stage_general_kernel<T, 6><<<(unsigned)blocks, threads, 0, st>>>(A, L); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_stage_general<float>(const StageArgs<float>&, int, const BoxList&, cudaStream_t);
template cudaError_t launch_stage_general<double>(const StageArgs<double>&, int, const BoxList&, cudaStream_t);

}  // namespace sbp
