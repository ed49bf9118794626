// Energy reduction for callers that cannot allocate device memory.
//
// The kernels are the same as sbp_energy's (launch_energy); only the scratch
// differs.  sbp_energy keeps its partial sums in a buffer the library obtains
// with cudaMalloc when the grid is bound.  Here the partial sums, the result
// and a status word live in one file-scope device array, so a call performs no
// allocation at all.  The array exists once per device that loads the library
// and is held until the process exits.
#include <math.h>
#include <string.h>

#include <mutex>

#include "launch.h"
#include "sbp.h"

namespace sbp {
void set_last_error(const char* msg);  // api.cu: the message sbp_last_error() returns
}

namespace {

constexpr int kMaxPartials = 4096;      // largest accepted nblocks
constexpr int kDefaultPartials = 1184;  // what sbp_energy uses (152 SMs x 8)
constexpr int kMaxDevices = 64;

// [0, kMaxPartials): per-block partial sums; [kMaxPartials]: the energy;
// [kMaxPartials + 1]: status bits (low 32 bits of the slot).  32.8 KB per device.
static __device__ __align__(256) double g_energy_scratch[kMaxPartials + 2];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

int reject(int code, const char* msg) {
  sbp::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int sbp_energy_noalloc(const void* q, const void* mat, int32_t nq, int32_t nr, int32_t ns, int64_t ldq,
                                  int64_t fs, int32_t order, int32_t precision, int32_t nblocks, double* out,
                                  void* stream) {
  if (!q || !mat || !out) return reject(SBP_ERR_ARG, "null input or output pointer");
  if (order != 2 && order != 4 && order != 6) return reject(SBP_ERR_ARG, "order must be 2, 4 or 6");
  if (precision != 32 && precision != 64) return reject(SBP_ERR_ARG, "precision must be 32 or 64");
  int32_t nmin = 0;
  sbp_min_nodes(order, &nmin);
  if (nq < nmin || nr < nmin || ns < nmin) return reject(SBP_ERR_ARG, "too few nodes for this order");
  if (ldq < nq || fs < ldq * (int64_t)nr * ns || fs >= (1LL << 31))
    return reject(SBP_ERR_ARG, "layout must satisfy nq <= ldq, ldq*nr*ns <= fs < 2^31");
  if (nblocks < 0 || nblocks > kMaxPartials)
    return reject(SBP_ERR_ARG, "nblocks must lie in 0..4096 (the static scratch holds 4096 partial sums)");
  if (nblocks == 0) nblocks = kDefaultPartials;

  // Once per device, with that device current: the device address of the scratch.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return reject(SBP_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return reject(SBP_ERR_UNSUPPORTED, "device index above 63");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_energy_scratch);
      if (e != cudaSuccess) return reject(SBP_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  double* partial = (double*)base;
  double* result = partial + kMaxPartials;
  unsigned* status = (unsigned*)(partial + kMaxPartials + 1);
  cudaStream_t st = (cudaStream_t)stream;

  // the status word must start at zero; partials and result are overwritten by this call
  e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return reject(SBP_ERR_CUDA, cudaGetErrorString(e));
  const sbp::Dims d{nq, nr, ns, (int)ldq, (int)(ldq * nr), fs};
  e = precision == 32 ? sbp::launch_energy<float>((const float*)q, (const float*)mat, d, order, partial, nblocks,
                                                  result, status, st)
                      : sbp::launch_energy<double>((const double*)q, (const double*)mat, d, order, partial,
                                                   nblocks, result, status, st);
  if (e != cudaSuccess) return reject(SBP_ERR_CUDA, cudaGetErrorString(e));
  double host[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(host, result, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return reject(SBP_ERR_CUDA, cudaGetErrorString(e));
  *out = host[0];
  unsigned bits = 0;
  memcpy(&bits, &host[1], sizeof(unsigned));
  if (bits != 0 || !isfinite(host[0])) return reject(SBP_ERR_NONFINITE, "energy is not finite");
  return SBP_OK;
}
