// Descriptors of the fifth-generation tensor-core MMA (tcgen05.mma, sm_100 family), packed
// from the field tables of the PTX ISA (tcgen05 "shared memory descriptor" and "instruction
// descriptor for .kind::f16").  Plain constexpr host/device code so that the packing can be
// checked on a CPU against the field table before any launch.
#pragma once

#include <stdint.h>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#define __device__
#endif
#endif

namespace sbp_umma {

// Swizzle modes of the shared-memory descriptor (bits 61-63).
constexpr uint32_t kSwizzleNone = 0, kSwizzle128B = 2, kSwizzle64B = 4, kSwizzle32B = 6;

// Shared-memory matrix descriptor (64 bits):
//   bits  0-13  start address >> 4 (shared window address)
//   bits 16-29  leading-dimension byte offset >> 4
//   bits 32-45  stride-dimension byte offset >> 4
//   bits 46-48  fixed value 0b001
//   bits 49-51  base offset (0: every swizzle pattern starts on its repeat boundary)
//   bit  52     leading-dimension mode (0: relative byte offset)
//   bits 61-63  swizzle mode
__host__ __device__ constexpr uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t swizzle) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)(swizzle & 7u) << 61);
}

// Instruction descriptor of tcgen05.mma .kind::f16 (32 bits), dense, no negation:
//   bits  4-5   D format (1: F32)
//   bits  7-9   A format (0: F16, 1: BF16)
//   bits 10-12  B format (0: F16, 1: BF16)
//   bit  15     A major (0: K-major, 1: MN-major)
//   bit  16     B major (0: K-major, 1: MN-major)
//   bits 17-22  N >> 3
//   bits 24-28  M >> 4
__host__ __device__ constexpr uint32_t instr_desc_bf16_f32(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Operand tiles of the GEMM as TMA writes them with 128-byte swizzling (bf16, 64-element rows of
// 128 bytes, 8-row swizzle atoms of 1024 bytes):
//  * K-major tile (rows x 64 k, one box): row r at r * 128 bytes.  Descriptor stride offset
//    1024 (next 8 rows); leading offset unused (16); the k-th group of 16 k starts 32 k bytes on.
//  * MN-major tile (64 k x rows, boxes of 64 rows side by side, 8192 bytes each): k row at
//    k * 128 bytes within a box.  Stride offset 1024 (next 8 k), leading offset 8192 (next 64
//    rows); the k-th group of 16 k starts 2048 k bytes on.
constexpr uint32_t kAtomBytes = 1024;
constexpr uint32_t kMnBoxBytes = 64 * 64 * 2;
__host__ __device__ constexpr uint64_t kmajor_desc(uint32_t tile_addr, int k16) {
  return smem_desc(tile_addr + 32u * (uint32_t)k16, 16, kAtomBytes, kSwizzle128B);
}
__host__ __device__ constexpr uint64_t mnmajor_desc(uint32_t tile_addr, int k16) {
  return smem_desc(tile_addr + 2048u * (uint32_t)k16, kMnBoxBytes, kAtomBytes, kSwizzle128B);
}

}  // namespace sbp_umma
