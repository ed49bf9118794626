// Host-side launchers of the kernels (defined in the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adjoint_args.h"
#include "common.cuh"
#include "tma.cuh"

namespace sbp {

// General adjoint stage: the prep kernel (Wb_k, yhat) and the one-thread-per-node L^T and
// gradient kernel; launch_adjoint_prep alone runs the first of the two.
template <typename T>
cudaError_t launch_adjoint(const AdjArgs<T>& A, int order, cudaStream_t st);
template <typename T>
cudaError_t launch_adjoint_prep(const AdjArgs<T>& A, int order, cudaStream_t st);

template <typename T>
cudaError_t launch_misfit(const T* q, const Dims& d, const int32_t* off, int n, int nb, long long bstride,
                          const double* data, double w, double* acc, T* ubar, cudaStream_t st);

template <typename T>
cudaError_t launch_stage_general(const StageArgs<T>& A, int order, const BoxList& L, cudaStream_t st);

// Tiled stage kernel over the whole grid, tile data by TMA through the tensor maps in
// `tm`; A.sclose must hold 2 b 6 planes per state.
template <typename T>
cudaError_t launch_stage_tiled(const StageArgs<T>& A, int order, const TmaSet& tm, cudaStream_t st);

// The tiled kernel's adjoint passes (after launch_adjoint_prep): pass 2, the material
// gradient on q = U_k (tensor maps of U_k), then pass 1, L^T on q = yhat (maps of yhat),
// which replaces Wb_k by A_k Wb_k.  A.nb members (tensor maps over all of them); the members
// add their gradients into the one shared gradient.
template <typename T>
cudaError_t launch_adjoint_tiled(const StageArgs<T>& A, int order, int pass, const TmaSet& tm, cudaStream_t st);

// One bounded mbarrier wait that nothing completes (sets status bit 8 after `polls` polls).
cudaError_t launch_wait_selftest(unsigned polls, unsigned* status, cudaStream_t st);

cudaError_t launch_metrics(const double* xyz, double* jmet, const Dims& d, int order, unsigned* status,
                           cudaStream_t st, SlabS sl = SlabS{});

template <typename T>
cudaError_t launch_material(const double* jmet, const double* rlm, T* met, T* mat, const Dims& d,
                            unsigned* status, cudaStream_t st);

// Largest relative departure of jmet (FP64 metrics) from a topography map: over all nodes,
// max(|a_q,y|, |a_q,z|, |a_r,x|, |a_r,z|) / |a_q,x| and |a_r,y - c a_q,x| / |a_r,y|, as the
// bits of a non-negative double, atomically maximised into *dev (zero it first; NaN counts as
// infinity).
cudaError_t launch_topography_check(const double* jmet, const Dims& d, double c, unsigned long long* dev,
                                    cudaStream_t st);

// Energy: per-block FP64 partial sums into partial[0..nblocks), then a single
// block sums them in a fixed order into *out (device).
template <typename T>
cudaError_t launch_energy(const T* q, const T* mat, const Dims& d, int order, double* partial,
                          int nblocks, double* out, unsigned* status, cudaStream_t st, SlabS sl = SlabS{});
int energy_blocks();

template <typename T>
cudaError_t launch_source(T* qout, T* dq, const Dims& d, const long long* off, const double* wsrc,
                          int nnodes, double gdt, double rk_b, int mode, cudaStream_t st);

template <typename T>
cudaError_t launch_receivers(const T* q, const Dims& d, const int32_t* off, int n, int nb, long long bstride,
                             T* traces, int n_t, long long step, cudaStream_t st);

// The interface trace of one face (v, sigma n, Z_p, Z_s at each face node and member), 8 nb face
// arrays in trace (see interface_trace_kernel).
template <typename T>
cudaError_t launch_interface_trace(const T* q, const T* met, const T* mat, const Dims& d, int face, int nb,
                                   long long bstride, T* trace, cudaStream_t st);

// FP64 fused multiply-add rate probe: one warm-up and one timed launch of `blocks` x 256 threads,
// 16 iters flops per thread; the timed launch's milliseconds in *ms.
cudaError_t probe_fp64_fma(int iters, int blocks, double* sink, float* ms, cudaStream_t st);

// Nearest node to each of n target points (3 FP64 values each, device) among the nodes of
// face `face` (0..5) or of the whole grid (face < 0), from the node coordinates xyz (3 FP64
// fields, device).  best, index: n device words each (scratch); index[r] receives the linear
// [s][r][q] node index of target r (smallest index among nodes at exactly the same distance).
cudaError_t launch_locate(const double* xyz, const Dims& d, int face, const double* targets, int n,
                          unsigned long long* best, unsigned long long* index, cudaStream_t st);

}  // namespace sbp
