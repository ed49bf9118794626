// Host-side launchers of the kernels (defined in the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "tma.cuh"

namespace sbp {

template <typename T>
cudaError_t launch_stage_general(const StageArgs<T>& A, int order, const BoxList& L, cudaStream_t st);

// Tiled interior kernel over `box` (q-start a multiple of 4), tile data by TMA through
// the tensor maps in `tm` (returns cudaErrorNotSupported when the box is empty).
template <typename T>
cudaError_t launch_stage_interior(const StageArgs<T>& A, int order, const Box& box, const TmaSet& tm,
                                  cudaStream_t st);

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
cudaError_t launch_source(T* qout, T* dq, const Dims& d, const int32_t* off, const double* wsrc,
                          int nnodes, double gdt, double rk_b, int mode, cudaStream_t st);

template <typename T>
cudaError_t launch_receivers(const T* q, const Dims& d, const int32_t* off, int n, T* traces,
                             int n_t, long long step, cudaStream_t st);

}  // namespace sbp
