// Host-side launchers of the kernels (defined in the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "tma.cuh"

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
  int bc_kind[6];
  T bc_gamma[6];
  T inv_h[3];
  T inv_h0[3];
};

// General adjoint stage: the prep kernel (Wb_k, yhat) and the one-thread-per-node L^T and
// gradient kernel; launch_adjoint_prep alone runs the first of the two.
template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T>& A, int order, cudaStream_t st);
template <typename T>
cudaError_t launch_adjoint_prep(const AdjArgs<T>& A, int order, cudaStream_t st);

template <typename T>
cudaError_t launch_misfit(const T* q, const Dims& d, const int32_t* off, int n, const double* data, double w,
                          double* acc, T* ubar, cudaStream_t st);

template <typename T>
cudaError_t launch_stage_general(const StageArgs<T>& A, int order, const BoxList& L, cudaStream_t st);

// Tiled stage kernel over the whole grid, tile data by TMA through the tensor maps in
// `tm`; A.sclose must hold 2 b 6 planes per state.
template <typename T>
cudaError_t launch_stage_tiled(const StageArgs<T>& A, int order, const TmaSet& tm, cudaStream_t st);

// The tiled kernel's adjoint passes (after launch_adjoint_prep): pass 2, the material
// gradient on q = U_k (tensor maps of U_k), then pass 1, L^T on q = yhat (maps of yhat),
// which replaces Wb_k by A_k Wb_k.  Unbatched grids only.
template <typename T>
cudaError_t launch_adjoint_tiled(const StageArgs<T>& A, int order, int pass, const TmaSet& tm, cudaStream_t st);

// One bounded mbarrier wait that nothing completes (sets status bit 8 after `polls` polls).
cudaError_t launch_wait_selftest(unsigned polls, unsigned* status, cudaStream_t st);

cudaError_t launch_metrics(const double* xyz, double* jmet, const Dims& d, int order, unsigned* status,
                           cudaStream_t st);

template <typename T>
cudaError_t launch_material(const double* jmet, const double* rlm, T* met, T* mat, const Dims& d,
                            unsigned* status, cudaStream_t st);

// Energy: per-block FP64 partial sums into partial[0..nblocks), then a single
// block sums them in a fixed order into *out (device).
template <typename T>
cudaError_t launch_energy(const T* q, const T* mat, const Dims& d, int order, double* partial,
                          int nblocks, double* out, unsigned* status, cudaStream_t st);
int energy_blocks();

template <typename T>
cudaError_t launch_source(T* qout, T* dq, const Dims& d, const long long* off, const double* wsrc,
                          int nnodes, double gdt, double rk_b, int mode, cudaStream_t st);

template <typename T>
cudaError_t launch_receivers(const T* q, const Dims& d, const int32_t* off, int n, int nb, long long bstride,
                             T* traces, int n_t, long long step, cudaStream_t st);

}  // namespace sbp
