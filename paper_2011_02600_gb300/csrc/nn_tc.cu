// BF16 GEMM on the fifth-generation tensor cores (tcgen05) for the surrogate network:
//     C[M x N] = beta C + op(A)[M x K] op(B)[K x N] (+ bias[m]) (ReLU)
// with the conventions of sbp_nn_gemm (row-major storage; op(A) = A stored M x K, or A^T with A
// stored K x M; op(B) = B stored K x N, or B^T with B stored N x K).
//
// One CTA of 128 threads computes a 128 x 256 tile of C:
//  * thread 0 streams 64-deep K slices of both operands into a ring of shared-memory stages
//    with 2D TMA loads (128-byte swizzle), in each operand's own orientation: K-major when k is
//    the contiguous index, MN-major otherwise; an mbarrier per stage counts the bytes;
//  * thread 32 issues tcgen05.mma (kind::f16, BF16 operands from shared memory through matrix
//    descriptors, FP32 accumulator of 128 lanes x 256 columns in tensor memory), four per slice
//    (K = 16 each), and frees each stage with tcgen05.commit on the stage's "empty" mbarrier;
//  * after the last slice a commit on the accumulator barrier releases the epilogue: each warp
//    reads its 32 accumulator rows with tcgen05.ld, transposes them through shared memory so
//    that a store instruction covers 32 consecutive columns of one row, adds the bias, applies
//    ReLU and stores FP32 or BF16 (FP32 atomics when K is split over CTAs).
// Every mbarrier wait is bounded: on a timeout the CTA records it in a device status word
// (sbp_nn_status), skips its stores, and still frees its tensor memory before it exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "sbp.h"
#include "tma.cuh"
#include "umma_desc.h"

namespace sbp_tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 2, THREADS = 128;
constexpr int A_BYTES = BM * BK * 2;              // 16 KB
constexpr int B_BYTES = BN * BK * 2;              // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;    // 48 KB, a multiple of the 1 KB swizzle atom
constexpr int TMEM_COLS = BN;                     // FP32 accumulator: one column per n
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* alignment slack */ + 256 /* barriers */;
constexpr unsigned kWaitLimit = 1u << 24;         // polls of about 64 ns: roughly a second

__device__ unsigned g_tc_status;  // bit 1: a wait timed out

struct Maps {
  CUtensorMap a, b;
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(sbp::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(sbp::smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   sbp::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 accumulator columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// A_MN / B_MN: operand stored MN-major (the m or n index contiguous) rather than K-major.
template <bool A_MN, bool B_MN>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ Maps maps, int M, int N, int K, int k_per, void* C, long long ldc,
                   int c_bf16, const float* __restrict__ bias, int relu, float beta) {
  extern __shared__ unsigned char smem_raw[];
  // stages at the first 1 KB boundary (the swizzle pattern repeats every 1 KB), barriers after
  unsigned char* base = smem_raw + ((1024u - (sbp::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  int* fail = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int kb = blockIdx.z * k_per;
  const int ke = min(K, kb + k_per);
  const int nk = (ke - kb + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      sbp::mbar_init(reinterpret_cast<unsigned long long*>(&full[s]), 1);
      sbp::mbar_init(reinterpret_cast<unsigned long long*>(&empty[s]), 1);
    }
    sbp::mbar_init(reinterpret_cast<unsigned long long*>(accum), 1);
    *fail = 0;
    sbp::fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbp::smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    // producer: TMA loads of the K slices
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES, use = kt / STAGES;
      if (use > 0 && !sbp::mbar_wait_bounded(reinterpret_cast<unsigned long long*>(&empty[s]), (use - 1) & 1,
                                            kWaitLimit)) {
        atomicOr(fail, 1);
        break;
      }
      unsigned char* st = base + s * STAGE_BYTES;
      sbp::mbar_expect_tx(reinterpret_cast<unsigned long long*>(&full[s]), STAGE_BYTES);
      const int k0 = kb + kt * BK;
      if (A_MN) {
        tma_load_2d(st, &maps.a, m0, k0, &full[s]);
        tma_load_2d(st + sbp_umma::kMnBoxBytes, &maps.a, m0 + 64, k0, &full[s]);
      } else {
        tma_load_2d(st, &maps.a, k0, m0, &full[s]);
      }
      unsigned char* sb = st + A_BYTES;
      if (B_MN) {
#pragma unroll
        for (int c = 0; c < BN / 64; ++c) tma_load_2d(sb + c * sbp_umma::kMnBoxBytes, &maps.b, n0 + 64 * c, k0, &full[s]);
      } else {
        tma_load_2d(sb, &maps.b, k0, n0, &full[s]);
      }
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer
    constexpr uint32_t idesc = sbp_umma::instr_desc_bf16_f32(BM, BN, A_MN, B_MN);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES, use = kt / STAGES;
      if (!sbp::mbar_wait_bounded(reinterpret_cast<unsigned long long*>(&full[s]), use & 1, kWaitLimit)) {
        atomicOr(fail, 1);
        break;
      }
      fence_after_sync();
      const uint32_t sa = sbp::smem_u32(base + s * STAGE_BYTES);
      const uint32_t sb = sa + A_BYTES;
#pragma unroll
      for (int k16 = 0; k16 < BK / 16; ++k16) {
        const uint64_t ad = A_MN ? sbp_umma::mnmajor_desc(sa, k16) : sbp_umma::kmajor_desc(sa, k16);
        const uint64_t bd = B_MN ? sbp_umma::mnmajor_desc(sb, k16) : sbp_umma::kmajor_desc(sb, k16);
        mma_bf16(tmem, ad, bd, idesc, (kt > 0 || k16 > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
    }
    mma_commit(accum);  // arrives when every MMA issued above has completed
  }

  // epilogue: all four warps, 32 accumulator rows each
  if (!sbp::mbar_wait_bounded(reinterpret_cast<unsigned long long*>(accum), 0, kWaitLimit)) atomicOr(fail, 1);
  fence_after_sync();
  __syncthreads();
  const bool ok = *fail == 0 && nk > 0;
  if (!ok && threadIdx.x == 0 && *fail) atomicOr(&g_tc_status, 1u);
  if (ok) {
    // Each warp moves its 32 accumulator rows out 32 columns at a time: tcgen05.ld gives one row
    // per thread; the warp transposes the 32 x 32 block through its own padded shared-memory
    // tile (the stage buffers are free once the accumulator barrier has passed) and then writes
    // one row per instruction, 32 consecutive columns across the lanes (128-byte segments).
    float* tile = reinterpret_cast<float*>(base) + warp * (32 * 33);
    const bool split = gridDim.z > 1;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      const int nb = n0 + 32 * c;
      if (nb >= N) break;  // uniform over the CTA
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * c), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = v[j];
      __syncwarp();
      const int n = nb + lane;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int m = m0 + warp * 32 + r;
        if (m >= M) break;  // uniform over the warp
        float x = tile[r * 33 + lane] + ((bias && blockIdx.z == 0) ? bias[m] : 0.f);
        if (n < N) {
          const long long idx = (long long)m * ldc + n;
          if (split) {
            atomicAdd((float*)C + idx, x);
          } else if (c_bf16) {
            if (relu) x = fmaxf(x, 0.f);
            ((__nv_bfloat16*)C)[idx] = __float2bfloat16(x);
          } else {
            if (beta != 0.f) x += beta * ((const float*)C)[idx];
            if (relu) x = fmaxf(x, 0.f);
            ((float*)C)[idx] = x;
          }
        }
      }
      __syncwarp();
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 2D tensor map of a row-major bf16 matrix with `rows` rows of `cols` elements (row pitch ld),
// box of box_cols x box_rows, 128-byte swizzle, zero fill outside the matrix.
bool encode(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld, int box_cols,
            int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace sbp_tc

namespace sbp_nn {
// Launch the tcgen05 GEMM; returns cudaErrorNotSupported when the operands do not suit TMA
// (leading dimensions not multiples of 8 elements, bases not 16-byte aligned).
cudaError_t launch_gemm_tc(int M, int N, int K, const void* A, long long lda, int ta, const void* B, long long ldb,
                           int tb, void* C, long long ldc, int c_bf16, const float* bias, int relu, float beta,
                           int sms, cudaStream_t st) {
  using namespace sbp_tc;
  if (lda % 8 || ldb % 8 || (uintptr_t)A % 16 || (uintptr_t)B % 16) return cudaErrorNotSupported;
  Maps maps;
  // A: op(A) = A (M x K, K-major) or A^T (A stored K x M, MN-major)
  const bool okA = ta ? encode(&maps.a, A, K, M, lda, 64, BK) : encode(&maps.a, A, M, K, lda, BK, BM);
  // B: op(B) = B (stored K x N, MN-major) or B^T (B stored N x K, K-major)
  const bool okB = tb ? encode(&maps.b, B, N, K, ldb, BK, BN) : encode(&maps.b, B, K, N, ldb, 64, BK);
  if (!okA || !okB) return cudaErrorInvalidValue;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, 1);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  int k_per = K;
  const long long tiles = (long long)grid.x * grid.y;
  const long long slots = 2LL * sms;  // two CTAs per SM (smem and tensor memory allow two)
  if (!c_bf16 && !relu && beta == 0.f && tiles < slots && K >= 8 * BK) {
    long long splits = (slots + tiles - 1) / tiles;
    splits = splits < K / (4 * BK) ? splits : K / (4 * BK);
    if (splits > 1) {
      k_per = (int)(((K + splits - 1) / splits + BK - 1) / BK * BK);
      grid.z = (unsigned)((K + k_per - 1) / k_per);
    }
  }
  cudaError_t e = cudaSuccess;
  if (grid.z > 1) {
    e = ldc == N ? cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * N, st)
                 : cudaMemset2DAsync(C, sizeof(float) * (size_t)ldc, 0, sizeof(float) * (size_t)N, (size_t)M, st);
    if (e != cudaSuccess) return e;
  }
  auto launch = [&](auto kern) -> cudaError_t {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (r != cudaSuccess) return r;
    kern<<<grid, THREADS, SMEM_BYTES, st>>>(maps, M, N, K, k_per, C, ldc, c_bf16, bias, relu, beta);
    return cudaGetLastError();
  };
  const bool a_mn = ta != 0, b_mn = tb == 0;
  if (a_mn && b_mn) return launch(gemm_tc_kernel<true, true>);
  if (a_mn) return launch(gemm_tc_kernel<true, false>);
  if (b_mn) return launch(gemm_tc_kernel<false, true>);
  return launch(gemm_tc_kernel<false, false>);
}

// Read and clear the tcgen05 GEMM's status word (synchronises the device).
cudaError_t gemm_tc_status(unsigned* bits) {
  unsigned v = 0, zero = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, sbp_tc::g_tc_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(sbp_tc::g_tc_status, &zero, sizeof(unsigned));
  if (e == cudaSuccess) *bits = v;
  return e;
}
}  // namespace sbp_nn
