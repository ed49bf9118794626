// Tensor-memory-accelerator (TMA) tile loads and mbarrier helpers (sm_90+ PTX),
// used by the interior stage kernel.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace sbp {

// Tensor maps of one interior-stage launch: the state with a halo on q and r, the
// three metric vectors (q-halo, r-halo, centre), the coefficients (centre), and a_q,x with
// halos on q and r (the topography-map variant's only metric read with a halo).
struct TmaSet {
  CUtensorMap state;
  CUtensorMap met_q;
  CUtensorMap met_r;
  CUtensorMap met_s;
  CUtensorMap mat;
  CUtensorMap met_j;
  CUtensorMap dq;  // the Runge-Kutta register (centre; the topography-map variant's stages)
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses (made visible to it
// by a barrier) before later async-proxy (TMA) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `limit` polls (with a short
// sleep between them) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned phase, unsigned limit) {
  for (unsigned n = 0; n < limit; ++n) {
    if (mbar_try_wait(bar, phase)) return true;
    __nanosleep(64);
  }
  return false;
}

// 4D tiled TMA load of one box into shared memory, completion on an mbarrier.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace sbp
