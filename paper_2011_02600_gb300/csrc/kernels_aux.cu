// Setup kernels (metrics, material) and the small per-step kernels (energy,
// source, receivers).
#include <math.h>

#include "common.cuh"
#include "launch.h"
#include "topo_check.h"

namespace sbp {

// ---------------------------------------------------------------------------
// Section 2.2: J and a[xi][eta] = J xi_eta from node coordinates, FP64, one thread per node
// (metrics_at in common.cuh).
template <int O>
__global__ void metrics_kernel(const double* __restrict__ xyz, double* __restrict__ jmet, Dims d, SlabS sl,
                               unsigned* status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nq * d.nr * (d.ns - sl.ghost_lo - sl.ghost_hi)) return;
  if (!metrics_at<O>(xyz, jmet, d, t, sl)) atomicOr(status, 2u);
}

cudaError_t launch_metrics(const double* xyz, double* jmet, const Dims& d, int order, unsigned* status,
                           cudaStream_t st, SlabS sl) {
  const long long total = (long long)d.nq * d.nr * (d.ns - sl.ghost_lo - sl.ghost_hi);
  const unsigned blocks = (unsigned)((total + 255) / 256);
  switch (order) {
    case 2: metrics_kernel<2><<<blocks, 256, 0, st>>>(xyz, jmet, d, sl, status); break;
    case 4: metrics_kernel<4><<<blocks, 256, 0, st>>>(xyz, jmet, d, sl, status); break;
    case 6: metrics_kernel<6><<<blocks, 256, 0, st>>>(xyz, jmet, d, sl, status); break;
    case 3: metrics_kernel<3><<<blocks, 256, 0, st>>>(xyz, jmet, d, sl, status); break;
    case 5: metrics_kernel<5><<<blocks, 256, 0, st>>>(xyz, jmet, d, sl, status); break;
    case 7: metrics_kernel<7><<<blocks, 256, 0, st>>>(xyz, jmet, d, sl, status); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Is the map a topography map (x = L_x q, y = L_y r, z = z(q, r, s))?  The largest deviation
// over all nodes (topography_deviation in topo_check.h).
__global__ void topography_check_kernel(const double* __restrict__ jmet, Dims d, double c,
                                        unsigned long long* dev) {
  const long long total = (long long)d.nq * d.nr * d.ns;
  double worst = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    worst = fmax(worst, topography_deviation(jmet, d, c, t));
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dev, (unsigned long long)__double_as_longlong(worst));
}

cudaError_t launch_topography_check(const double* jmet, const Dims& d, double c, unsigned long long* dev,
                                    cudaStream_t st) {
  topography_check_kernel<<<1024, 256, 0, st>>>(jmet, d, c, dev);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Solver coefficients: met = a (cast), mat = (1/(rho J), lambda/J, mu/J).
template <typename T>
__global__ void material_kernel(const double* __restrict__ jmet, const double* __restrict__ rlm,
                                T* __restrict__ met, T* __restrict__ mat, Dims d, unsigned* status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)d.nq * d.nr * d.ns;
  if (t >= total) return;
  const int i = (int)(t % d.nq);
  const int j = (int)((t / d.nq) % d.nr);
  const int k = (int)(t / ((long long)d.nq * d.nr));
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const double J = jmet[n0];
#pragma unroll
  for (int c = 0; c < 9; ++c) met[c * d.fs + n0] = (T)jmet[(1 + c) * d.fs + n0];
  const double rho = rlm[n0], lam = rlm[d.fs + n0], mu = rlm[2 * d.fs + n0];
  mat[n0] = (T)(1.0 / (rho * J));
  mat[d.fs + n0] = (T)(lam / J);
  mat[2 * d.fs + n0] = (T)(mu / J);
  if (!(rho > 0.0) || !(mu > 0.0) || !(lam + 2.0 * mu > 0.0)) atomicOr(status, 4u);
  if (!(J > 0.0)) atomicOr(status, 2u);
}

template <typename T>
cudaError_t launch_material(const double* jmet, const double* rlm, T* met, T* mat, const Dims& d,
                            unsigned* status, cudaStream_t st) {
  const long long total = (long long)d.nq * d.nr * d.ns;
  material_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(jmet, rlm, met, mat, d, status);
  return cudaGetLastError();
}
template cudaError_t launch_material<float>(const double*, const double*, float*, float*, const Dims&,
                                            unsigned*, cudaStream_t);
template cudaError_t launch_material<double>(const double*, const double*, double*, double*,
                                             const Dims&, unsigned*, cudaStream_t);

// ---------------------------------------------------------------------------
// Energy (Eq. physical_energy_discrete with P~): 1/2 sum H J (rho |v|^2 + sigma^T S sigma),
// written with the stored coefficients: J rho = 1/(1/(rho J)), and
// J sigma^T S sigma = [sum s_ii^2 + 2 sum s_ij^2 - l/(3 l + 2 m) tr^2] / (2 m)
// with l = lambda/J, m = mu/J.  Accumulated in FP64 (per row, per thread, then warp
// shuffles and a fixed-order block reduction), so the result is deterministic.
constexpr int kEnergyBlocks = 1184;  // 152 SMs x 8
constexpr int kEnergyThreads = 256;
int energy_blocks() { return kEnergyBlocks; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One warp per (r, s) row of nodes (q contiguous, coalesced); rows strided over the grid.
// A slab of a decomposed block sums its own planes only, with the block's weights along s.
template <typename T, int O>
__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(const T* __restrict__ q, const T* __restrict__ mat,
                                                                Dims d, SlabS sl, double* __restrict__ partial,
                                                                unsigned* status) {
  const int warps = kEnergyThreads / 32;
  const int lane = threadIdx.x & 31;
  const int k0 = sl.ghost_lo, nown = d.ns - sl.ghost_lo - sl.ghost_hi;
  const int nsg = sl.ns_global > 0 ? sl.ns_global : d.ns;
  const int rows = d.nr * nown;
  const double hq = 1.0 / (d.nq - 1), hr = 1.0 / (d.nr - 1), hs = 1.0 / (nsg - 1);
  const long long fs = d.fs;
  double acc = 0.0;
  bool bad = false;
  for (int row = blockIdx.x * warps + (threadIdx.x >> 5); row < rows; row += gridDim.x * warps) {
    const int j = row % d.nr, k = k0 + row / d.nr;
    const double wjk = hr * norm_weight<O>(j, d.nr) * hs * norm_weight<O>(k + sl.k_offset, nsg);
    const long long base = (long long)k * d.plane + (long long)j * d.ldq;
    double racc = 0.0;
    for (int i = lane; i < d.nq; i += 32) {
      const long long n0 = base + i;
      T v[3], sg[6];
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = q[c * fs + n0];
#pragma unroll
      for (int c = 0; c < 6; ++c) sg[c] = q[(3 + c) * fs + n0];
      const T dens = energy_density<T>(v, sg, mat[n0], mat[fs + n0], mat[2 * fs + n0]);
      bad |= !isfinite(dens);
      racc += hq * norm_weight<O>(i, d.nq) * (double)dens;
    }
    acc += wjk * racc;
  }
  __shared__ double red[kEnergyThreads / 32];
  acc = warp_sum(acc);
  if (lane == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kEnergyThreads / 32 ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = 0.5 * v;
  }
  if (bad) atomicOr(status, 1u);
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) v += partial[t];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    w = warp_sum(w);
    if (threadIdx.x == 0) *out = w;
  }
}

template <typename T>
cudaError_t launch_energy(const T* q, const T* mat, const Dims& d, int order, double* partial, int nblocks,
                          double* out, unsigned* status, cudaStream_t st, SlabS sl) {
  switch (order) {
    case 2: energy_kernel<T, 2><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status); break;
    case 4: energy_kernel<T, 4><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status); break;
    case 6: energy_kernel<T, 6><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status); break;
    case 3: energy_kernel<T, 3><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status); break;
    case 5: energy_kernel<T, 5><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status); break;
    case 7: energy_kernel<T, 7><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status); break;
    case kTraditional + 2:
      energy_kernel<T, kTraditional + 2><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status);
      break;
    case kTraditional + 4:
      energy_kernel<T, kTraditional + 4><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status);
      break;
    case kTraditional + 6:
      energy_kernel<T, kTraditional + 6><<<nblocks, kEnergyThreads, 0, st>>>(q, mat, d, sl, partial, status);
      break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_partials_kernel<<<1, 1024, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}
template cudaError_t launch_energy<float>(const float*, const float*, const Dims&, int, double*, int, double*,
                                          unsigned*, cudaStream_t, SlabS);
template cudaError_t launch_energy<double>(const double*, const double*, const Dims&, int, double*, int,
                                           double*, unsigned*, cudaStream_t, SlabS);

// ---------------------------------------------------------------------------
// Point source: wsrc[n*6 + c] = -M_c delta_h at source node n; in a stage the
// stress rates gain g(t) * wsrc, i.e. dq += dt g w and qout += B dt g w
// (the stage update is linear in the rate).
template <typename T>
__global__ void source_kernel(T* __restrict__ qout, T* __restrict__ dq, Dims d, const long long* __restrict__ off,
                              const double* __restrict__ wsrc, int nnodes, double gdt, double rk_b, int mode) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnodes * 6) return;
  const int n = t / 6, c = t % 6;
  const long long idx = (long long)(3 + c) * d.fs + off[n];
  const double add = gdt * wsrc[t];
  if (mode == kModeRhs) {
    qout[idx] = (T)((double)qout[idx] + add);
    return;
  }
  dq[idx] = (T)((double)dq[idx] + add);
  qout[idx] = (T)((double)qout[idx] + rk_b * add);
}

template <typename T>
cudaError_t launch_source(T* qout, T* dq, const Dims& d, const long long* off, const double* wsrc, int nnodes,
                          double gdt, double rk_b, int mode, cudaStream_t st) {
  if (nnodes == 0) return cudaSuccess;
  source_kernel<T><<<(nnodes * 6 + 127) / 128, 128, 0, st>>>(qout, dq, d, off, wsrc, nnodes, gdt, rk_b, mode);
  return cudaGetLastError();
}
template cudaError_t launch_source<float>(float*, float*, const Dims&, const long long*, const double*, int,
                                          double, double, int, cudaStream_t);
template cudaError_t launch_source<double>(double*, double*, const Dims&, const long long*, const double*, int,
                                           double, double, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Interface trace of face `face` (xi = face / 2): at every node of the face and member b,
// trace[(8 b + c) n_face + face_index] = v (c = 0..2), T = sigma n (3..5) with n = a_xi / |a_xi|,
// Z_p, Z_s (6, 7) from the stored coefficients, for the other block's interface penalty.
template <typename T>
__global__ void interface_trace_kernel(const T* __restrict__ q, const T* __restrict__ met, const T* __restrict__ mat,
                                       Dims d, int face, int nb, long long bstride, T* __restrict__ trace) {
  const int xi = face / 2, side = face % 2;
  const long long nf = xi == 0 ? (long long)d.nr * d.ns : xi == 1 ? (long long)d.nq * d.ns : (long long)d.nq * d.nr;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf * nb) return;
  const int b = (int)(t / nf);
  const long long f = t % nf;
  const int na = xi == 0 ? d.nr : d.nq;   // the face's first (fastest) axis
  const int u = (int)(f % na), w = (int)(f / na);
  const int i = xi == 0 ? (side ? d.nq - 1 : 0) : u;
  const int j = xi == 0 ? u : xi == 1 ? (side ? d.nr - 1 : 0) : w;
  const int k = xi == 2 ? (side ? d.ns - 1 : 0) : w;
  const long long n0 = (long long)k * d.plane + (long long)j * d.ldq + i;
  const long long fs = d.fs;
  const T* qb = q + (long long)b * bstride;
  const T a[3] = {met[(3 * xi) * fs + n0], met[(3 * xi + 1) * fs + n0], met[(3 * xi + 2) * fs + n0]};
  const T ian = T(1) / sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  const T n[3] = {a[0] * ian, a[1] * ian, a[2] * ian};
  T sg[6], Tr[3];
#pragma unroll
  for (int c = 0; c < 6; ++c) sg[c] = qb[(3 + c) * fs + n0];
  flux(n, sg, Tr);
  const T irhoJ = mat[n0], lamJ = mat[fs + n0], muJ = mat[2 * fs + n0];
  T* out = trace + (long long)b * 8 * nf + f;
#pragma unroll
  for (int c = 0; c < 3; ++c) out[c * nf] = qb[c * fs + n0];
#pragma unroll
  for (int c = 0; c < 3; ++c) out[(3 + c) * nf] = Tr[c];
  out[6 * nf] = sqrt((lamJ + T(2) * muJ) / irhoJ);
  out[7 * nf] = sqrt(muJ / irhoJ);
}

template <typename T>
cudaError_t launch_interface_trace(const T* q, const T* met, const T* mat, const Dims& d, int face, int nb,
                                   long long bstride, T* trace, cudaStream_t st) {
  const int xi = face / 2;
  const long long nf = xi == 0 ? (long long)d.nr * d.ns : xi == 1 ? (long long)d.nq * d.ns : (long long)d.nq * d.nr;
  const long long total = nf * nb;
  interface_trace_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(q, met, mat, d, face, nb, bstride, trace);
  return cudaGetLastError();
}
template cudaError_t launch_interface_trace<float>(const float*, const float*, const float*, const Dims&, int, int,
                                                   long long, float*, cudaStream_t);
template cudaError_t launch_interface_trace<double>(const double*, const double*, const double*, const Dims&, int,
                                                    int, long long, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// Receivers: trace[b][r][c][step] = v_c of state b at the receiver node.
template <typename T>
__global__ void receivers_kernel(const T* __restrict__ q, Dims d, const int32_t* __restrict__ off, int n, int nb,
                                 long long bstride, T* __restrict__ traces, int n_t, long long step) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * n * 3 || step >= n_t) return;
  const int b = t / (3 * n), r = (t / 3) % n, c = t % 3;
  traces[(long long)t * n_t + step] = q[(long long)b * bstride + (long long)c * d.fs + off[r]];
}

template <typename T>
cudaError_t launch_receivers(const T* q, const Dims& d, const int32_t* off, int n, int nb, long long bstride,
                             T* traces, int n_t, long long step, cudaStream_t st) {
  if (n == 0 || step < 0 || step >= n_t) return cudaSuccess;
  receivers_kernel<T><<<(nb * n * 3 + 127) / 128, 128, 0, st>>>(q, d, off, n, nb, bstride, traces, n_t, step);
  return cudaGetLastError();
}
// ---------------------------------------------------------------------------
// Receivers by position: the node nearest (Euclidean, in the node coordinates xyz) to each
// target point, among the nodes of one face (0..5) or of the whole grid (face < 0).  Pass 1
// finds the smallest squared distance per target (atomicMin on the bits of a non-negative
// double, which order like the values); pass 2 takes the smallest node index at exactly that
// distance, so the choice is deterministic.
__device__ __forceinline__ long long locate_candidate(const Dims& d, int face, long long t) {
  // t-th candidate node as a linear [s][r][q] node index (not an offset)
  if (face < 0) return t;
  const int xi = face / 2;
  const int side = face % 2;
  const long long nq = d.nq, nr = d.nr, ns = d.ns;
  if (xi == 0) {  // (k, j) plane at i = 0 or nq - 1
    const long long j = t % nr, k = t / nr;
    return (k * nr + j) * nq + (side ? nq - 1 : 0);
  }
  if (xi == 1) {  // (k, i) plane at j = 0 or nr - 1
    const long long i = t % nq, k = t / nq;
    return (k * nr + (side ? nr - 1 : 0)) * nq + i;
  }
  return (long long)(side ? ns - 1 : 0) * nr * nq + t;  // (j, i) plane at k = 0 or ns - 1
}

__device__ __forceinline__ double locate_dist2(const double* __restrict__ xyz, const Dims& d, long long node,
                                               const double* __restrict__ target) {
  const long long i = node % d.nq, j = (node / d.nq) % d.nr, k = node / ((long long)d.nq * d.nr);
  const long long off = k * d.plane + j * d.ldq + i;
  const double dx = xyz[off] - target[0], dy = xyz[d.fs + off] - target[1], dz = xyz[2 * d.fs + off] - target[2];
  return dx * dx + dy * dy + dz * dz;
}

__global__ void locate_min_kernel(const double* __restrict__ xyz, Dims d, int face, long long ncand,
                                  const double* __restrict__ targets, unsigned long long* __restrict__ best) {
  const int r = blockIdx.y;
  const double* tg = targets + 3 * r;
  double m = 1.0 / 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ncand; t += (long long)gridDim.x * blockDim.x)
    m = fmin(m, locate_dist2(xyz, d, locate_candidate(d, face, t), tg));
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m < 1.0 / 0.0) atomicMin(best + r, (unsigned long long)__double_as_longlong(m));
}

__global__ void locate_index_kernel(const double* __restrict__ xyz, Dims d, int face, long long ncand,
                                    const double* __restrict__ targets, const unsigned long long* __restrict__ best,
                                    unsigned long long* __restrict__ index) {
  const int r = blockIdx.y;
  const double* tg = targets + 3 * r;
  const unsigned long long b = best[r];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ncand; t += (long long)gridDim.x * blockDim.x) {
    const long long node = locate_candidate(d, face, t);
    if ((unsigned long long)__double_as_longlong(locate_dist2(xyz, d, node, tg)) == b)
      atomicMin(index + r, (unsigned long long)node);
  }
}

cudaError_t launch_locate(const double* xyz, const Dims& d, int face, const double* targets, int n,
                          unsigned long long* best, unsigned long long* index, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const long long ncand = face < 0 ? (long long)d.nq * d.nr * d.ns
                          : face < 2 ? (long long)d.nr * d.ns : face < 4 ? (long long)d.nq * d.ns
                                                                         : (long long)d.nq * d.nr;
  cudaError_t e = cudaMemsetAsync(best, 0xff, sizeof(unsigned long long) * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(index, 0xff, sizeof(unsigned long long) * n, st);
  if (e != cudaSuccess) return e;
  const long long want = (ncand + 255) / 256;
  const dim3 grid((unsigned)(want < 1216 ? want : 1216), (unsigned)n);
  locate_min_kernel<<<grid, 256, 0, st>>>(xyz, d, face, ncand, targets, best);
  locate_index_kernel<<<grid, 256, 0, st>>>(xyz, d, face, ncand, targets, best, index);
  return cudaGetLastError();
}

template cudaError_t launch_receivers<float>(const float*, const Dims&, const int32_t*, int, int, long long, float*,
                                             int, long long, cudaStream_t);
template cudaError_t launch_receivers<double>(const double*, const Dims&, const int32_t*, int, int, long long,
                                              double*, int, long long, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 arithmetic rate probe: 8 independent fused multiply-add chains per thread (enough to
// cover the FP64 pipe's latency), no memory traffic; the result is written only if it takes an
// impossible value, so that the chains are not removed.
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, double seed, double* sink) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + 1e-3 * (threadIdx.x + 7 * c);
  const double b = 0.9999999, d = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == -1.0) sink[blockIdx.x] = s;
}

cudaError_t probe_fp64_fma(int iters, int blocks, double* sink, float* ms, cudaStream_t st) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_probe_kernel<<<blocks, 256, 0, st>>>(iters / 10 + 1, 1.0, sink);  // warm-up
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    fma_probe_kernel<<<blocks, 256, 0, st>>>(iters, 1.0, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace sbp
