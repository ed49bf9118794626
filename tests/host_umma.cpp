// Host build of csrc/umma_desc.h: the tcgen05 descriptor packing, for tests/test_host_umma.py.
#include <stdint.h>

#include "umma_desc.h"

extern "C" {
uint64_t host_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t swizzle) {
  return sbp_umma::smem_desc(addr, lbo, sbo, swizzle);
}
uint64_t host_kmajor_desc(uint32_t addr, int k16) { return sbp_umma::kmajor_desc(addr, k16); }
uint64_t host_mnmajor_desc(uint32_t addr, int k16) { return sbp_umma::mnmajor_desc(addr, k16); }
uint32_t host_instr_desc(int M, int N, int a_mn, int b_mn) {
  return sbp_umma::instr_desc_bf16_f32(M, N, a_mn != 0, b_mn != 0);
}
}
