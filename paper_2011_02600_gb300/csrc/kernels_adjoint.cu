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

#include "adjoint_node.cuh"
#include "adjoint_terms.cuh"
#include "common.cuh"
#include "launch.h"

namespace sbp {

// blockIdx.y: member of a batch of independent states.
template <typename T, int O>
__global__ void adjoint_prep_kernel(AdjArgs<T> A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)A.d.nq * A.d.nr * A.d.ns) return;
  adjoint_prep_at<T, O>(adjoint_member(A, blockIdx.y), t);
}

// One thread per node: L^T, the stage updates and the gradient (adjoint_node.cuh).
template <typename T, int O>
__global__ void __launch_bounds__(256) adjoint_stage_kernel(AdjArgs<T> A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)A.d.nq * A.d.nr * A.d.ns) return;
  adjoint_stage_at<T, O>(adjoint_member(A, blockIdx.y), t);
}

template <typename T>
cudaError_t launch_adjoint_prep(const AdjArgs<T>& A, int order, cudaStream_t st) {
  const long long total = (long long)A.d.nq * A.d.nr * A.d.ns;
  const dim3 blocks((unsigned)((total + 255) / 256), (unsigned)A.nb);
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
  const dim3 blocks((unsigned)((total + 255) / 256), (unsigned)A.nb);
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
// receivers that share a node each contribute their own source.  Thread t covers member
// t / (3 n) of a batch (its state, data, accumulators and ubar at member stride bstride).
template <typename T>
__global__ void misfit_kernel(const T* __restrict__ q, Dims d, const int32_t* __restrict__ off, int n, int nb,
                              long long bstride, const double* __restrict__ data, double w,
                              double* __restrict__ acc, T* ubar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 3 * nb) return;
  const int b = t / (3 * n), r = (t / 3) % n, c = t % 3;
  const long long idx = (long long)b * bstride + (long long)c * d.fs + off[r];
  const double diff = (double)q[idx] - data[t];
  if (acc) acc[t] += 0.5 * w * diff * diff;
  if (ubar) atomicAdd(&ubar[idx], (T)(w * diff));
}

template <typename T>
cudaError_t launch_misfit(const T* q, const Dims& d, const int32_t* off, int n, int nb, long long bstride,
                          const double* data, double w, double* acc, T* ubar, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  misfit_kernel<T><<<(n * 3 * nb + 127) / 128, 128, 0, st>>>(q, d, off, n, nb, bstride, data, w, acc, ubar);
  return cudaGetLastError();
}

template cudaError_t launch_adjoint<float>(const AdjArgs<float>&, int, cudaStream_t);
template cudaError_t launch_adjoint<double>(const AdjArgs<double>&, int, cudaStream_t);
template cudaError_t launch_adjoint_prep<float>(const AdjArgs<float>&, int, cudaStream_t);
template cudaError_t launch_adjoint_prep<double>(const AdjArgs<double>&, int, cudaStream_t);
template cudaError_t launch_misfit<float>(const float*, const Dims&, const int32_t*, int, int, long long,
                                          const double*, double, double*, float*, cudaStream_t);
template cudaError_t launch_misfit<double>(const double*, const Dims&, const int32_t*, int, int, long long,
                                           const double*, double, double*, double*, cudaStream_t);

}  // namespace sbp
