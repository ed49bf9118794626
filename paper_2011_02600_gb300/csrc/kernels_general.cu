// General stage kernel: one thread per node of a list of boxes; every row of
// D+ and D- (interior stencil or closure) read from global memory, the penalties
// of every face the node lies on, and the fused Runge-Kutta stage.  It computes
// the same scheme as the tiled kernel and serves to cross-check it
// (sbp_set_kernel_path(1)).
#include "common.cuh"
#include "launch.h"

namespace sbp {

template <typename T, int O>
__global__ void __launch_bounds__(256) stage_general_kernel(StageArgs<T> A, BoxList L) {
  // member blockIdx.y of a batch of independent states
  const long long boff = (long long)blockIdx.y * A.bstride;
  A.q += boff;
  A.qout += boff;
  if (A.mode != kModeRhs) A.dq += boff;
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
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const int pos[3] = {i, j, k};
  T rv[3], e[6], qc[9];
  raw_operator_at<T, O>(A.q, A.met, A.mat, d, n0, pos, A.inv_h, A.inv_h0, A.bc_kind, A.bc_gamma, rv, e, qc, &A.ifc,
                        (int)blockIdx.y);
  const T irhoJ = A.mat[n0], lamJ = A.mat[d.fs + n0], muJ = A.mat[2 * d.fs + n0];
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
  const dim3 grid((unsigned)blocks, (unsigned)A.nb);
  switch (order) {
    case 2: stage_general_kernel<T, 2><<<grid, threads, 0, st>>>(A, L); break;
    case 4: stage_general_kernel<T, 4><<<grid, threads, 0, st>>>(A, L); break;
    case 6: stage_general_kernel<T, 6><<<grid, threads, 0, st>>>(A, L); break;
    case 3: stage_general_kernel<T, 3><<<grid, threads, 0, st>>>(A, L); break;
    case 5: stage_general_kernel<T, 5><<<grid, threads, 0, st>>>(A, L); break;
    case 7: stage_general_kernel<T, 7><<<grid, threads, 0, st>>>(A, L); break;
    case kTraditional + 2: stage_general_kernel<T, kTraditional + 2><<<grid, threads, 0, st>>>(A, L); break;
    case kTraditional + 4: stage_general_kernel<T, kTraditional + 4><<<grid, threads, 0, st>>>(A, L); break;
    case kTraditional + 6: stage_general_kernel<T, kTraditional + 6><<<grid, threads, 0, st>>>(A, L); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_stage_general<float>(const StageArgs<float>&, int, const BoxList&, cudaStream_t);
template cudaError_t launch_stage_general<double>(const StageArgs<double>&, int, const BoxList&, cudaStream_t);

}  // namespace sbp
