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

#include <cudaTypedefs.h>

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

// Set-up state per device: the scratch's device address and the unique id of the context it
// was looked up in.  A device reset (cudaDeviceReset) ends that context; the next call finds a
// different id, looks the address up again and does not use the stale one.
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  void* addr = nullptr;
};
std::mutex g_setup_mutex;
ScratchSlot g_scratch[kMaxDevices];

// Unique id of the calling thread's current context (driver API through the runtime's
// entry-point query, so that the library needs no link against libcuda); 0 if there is none.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (PFN_cuCtxGetCurrent_v4000)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (PFN_cuCtxGetId_v12000)p;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

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

  // Set-up, once per device (and again after a device reset), with that device current: the
  // device address of the scratch.  Host code cannot use g_energy_scratch itself as an address.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return reject(SBP_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return reject(SBP_ERR_UNSUPPORTED, "device index above 63");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchSlot& slot = g_scratch[dev];
    const unsigned long long id = current_context_id();
    if (!slot.addr || id == 0 || id != slot.ctx_id) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_energy_scratch);  // creates the context if there was none yet
      if (e != cudaSuccess) return reject(SBP_ERR_CUDA, cudaGetErrorString(e));
      slot.addr = p;
      slot.ctx_id = current_context_id();
    }
    base = slot.addr;
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
