// BF16 GEMM on the fifth-generation tensor cores (tcgen05) for the surrogate network:
//     C[M x N] = beta C + op(A)[M x K] op(B)[K x N] (+ bias[m]) (ReLU)
// with the conventions of sbp_nn_gemm (row-major storage; op(A) = A stored M x K, or A^T with A
// stored K x M; op(B) = B stored K x N, or B^T with B stored N x K).
//
// A persistent kernel, one CTA of ten warps per SM, takes 128 x 256 tiles of C in turn:
//  * warp 0 (one thread) streams 64-deep K slices of both operands into a ring of four
//    shared-memory stages with 2D TMA loads (128-byte swizzle), in each operand's own
//    orientation: K-major when k is the contiguous index, MN-major otherwise; an mbarrier per
//    stage counts the bytes, another frees the stage;
//  * warp 1 (one thread) issues tcgen05.mma (kind::f16, BF16 operands from shared memory
//    through matrix descriptors), four per slice (K = 16 each), into one of two FP32
//    accumulators of 128 lanes x 256 columns in tensor memory (all 512 columns), and frees each
//    stage with tcgen05.commit; a commit on the accumulator's barrier hands it to the epilogue;
//  * warps 2-9 drain the other accumulator meanwhile, two warps per group of 32 accumulator lanes
//    (half of the columns each): tcgen05.ld, bias and ReLU in registers, then a 32 x 32 box (FP32
//    or BF16) into swizzled shared memory and a TMA store (a TMA reduce-add when K is split over
//    work items), or, when C is accumulated into or does not suit TMA, a transpose through shared
//    memory and stores that cover 32 consecutive columns of a row; then an arrival that gives the
//    accumulator back to the MMA warp.
// Every mbarrier wait is bounded: on a timeout the CTA records it in a device status word
// (sbp_nn_status), its roles stop, and it still waits for its MMAs and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "sbp.h"
#include "tma.cuh"
#include "umma_desc.h"

namespace sbp_tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int EPI_WARPS = 8;                      // two per accumulator lane group, half the columns each
constexpr int WARPS = 2 + EPI_WARPS, THREADS = 32 * WARPS;  // producer, MMA issuer, epilogue warps
constexpr int A_BYTES = BM * BK * 2;              // 16 KB
constexpr int B_BYTES = BN * BK * 2;              // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;    // 48 KB, a multiple of the 1 KB swizzle atom
constexpr int ACC_COLS = BN;                      // FP32 accumulator: one column per n
constexpr int TMEM_COLS = 2 * ACC_COLS;           // two accumulators: the whole tensor memory
constexpr int EPI_WARP_BYTES = 4096;              // per epilogue warp: one 32 x 32 FP32 buffer
constexpr int SMEM_BYTES = 1024 /* alignment slack */ + STAGES * STAGE_BYTES + EPI_WARPS * EPI_WARP_BYTES + 256;
static_assert(SMEM_BYTES <= 232448, "shared memory per block");

// How the epilogue writes C: through the warp's transpose tile with plain stores (BF16 output or
// accumulation into C), or from swizzled shared-memory buffers by TMA (store, or reduce-add
// when K is split over work items).
enum EpiMode : int { kEpiDirect = 0, kEpiTmaStore = 1, kEpiTmaAdd = 2, kEpiTmaStoreBf16 = 3 };
constexpr unsigned kWaitLimit = 1u << 24;         // polls of about 64 ns: roughly a second

__device__ unsigned g_tc_status;  // bit 1: a wait timed out

struct Maps {
  CUtensorMap a, b, c;  // c: FP32 C with 32 x 32 boxes and 128-byte swizzle (TMA epilogue modes)
};

// TMA store (or reduce-add) of a 32 x 32 FP32 box from shared memory at C[y][x], as a bulk group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src, bool add) {
  if (add)
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(sbp::smem_u32(src))
                 : "memory");
  else
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(sbp::smem_u32(src))
                 : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sbp::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool wait(uint64_t* bar, unsigned parity) {
  return sbp::mbar_wait_bounded(reinterpret_cast<unsigned long long*>(bar), parity, kWaitLimit);
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

// Work item w (of tm x tn x splits).  m tiles fastest: the CTAs running at the same time share
// their B tiles (the larger operand) through L2, which suits a B larger than L2.  n tiles fastest
// (n_fast): one wave of CTAs reads every B tile once, from DRAM, and the later waves (the other m
// tiles) find B in L2 at L2 latency instead of all waiting together on the same DRAM reads.
struct Item {
  int m0, n0, kb, ke;
};
__device__ __forceinline__ Item item(int w, int tm, int tn, int k_per, int K, int n_fast) {
  Item it;
  const int per = tm * tn;
  const int z = w / per, r = w % per;
  it.m0 = (n_fast ? r / tn : r % tm) * BM;
  it.n0 = (n_fast ? r % tn : r / tm) * BN;
  it.kb = z * k_per;
  it.ke = min(K, it.kb + k_per);
  return it;
}

// Persistent kernel: CTA b takes work items b, b + gridDim.x, ...  A_MN / B_MN: operand stored
// MN-major (the m or n index contiguous) rather than K-major.
template <bool A_MN, bool B_MN>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ Maps maps, int M, int N, int K, int k_per, int tm, int tn, int items,
                   void* C, long long ldc, int c_bf16, const float* __restrict__ bias, int relu, float beta,
                   int epi_mode, int n_fast) {
  extern __shared__ unsigned char smem_raw[];
  // stages at the first 1 KB boundary (the swizzle pattern repeats every 1 KB), then the
  // epilogue warps' transpose tiles, then the barriers
  unsigned char* base = smem_raw + ((1024u - (sbp::smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* epi = base + STAGES * STAGE_BYTES;   // 1 KB aligned: the swizzled store buffers need it
  uint64_t* full = reinterpret_cast<uint64_t*>(epi + EPI_WARPS * EPI_WARP_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* fail = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      sbp::mbar_init(reinterpret_cast<unsigned long long*>(&full[s]), 1);
      sbp::mbar_init(reinterpret_cast<unsigned long long*>(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      sbp::mbar_init(reinterpret_cast<unsigned long long*>(&acc_full[b]), 1);
      sbp::mbar_init(reinterpret_cast<unsigned long long*>(&acc_empty[b]), 32 * EPI_WARPS);  // epilogue threads
    }
    sbp::mbar_init(reinterpret_cast<unsigned long long*>(done), 1);
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

  if (warp == 0) {
    if (lane == 0) {
      // producer: TMA loads of every K slice of every item, through the ring of stages
      int it = 0;
      for (int w = blockIdx.x; w < items && !*(volatile int*)fail; w += gridDim.x) {
        const Item I = item(w, tm, tn, k_per, K, n_fast);
        const int nk = (I.ke - I.kb + BK - 1) / BK;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % STAGES, use = it / STAGES;
          if (use > 0 && !wait(&empty[s], (use - 1) & 1)) {
            atomicOr(fail, 1);
            break;
          }
          unsigned char* st = base + s * STAGE_BYTES;
          sbp::mbar_expect_tx(reinterpret_cast<unsigned long long*>(&full[s]), STAGE_BYTES);
          const int k0 = I.kb + kt * BK;
          if (A_MN) {
            tma_load_2d(st, &maps.a, I.m0, k0, &full[s]);
            tma_load_2d(st + sbp_umma::kMnBoxBytes, &maps.a, I.m0 + 64, k0, &full[s]);
          } else {
            tma_load_2d(st, &maps.a, k0, I.m0, &full[s]);
          }
          unsigned char* sb = st + A_BYTES;
          if (B_MN) {
#pragma unroll
            for (int c = 0; c < BN / 64; ++c)
              tma_load_2d(sb + c * sbp_umma::kMnBoxBytes, &maps.b, I.n0 + 64 * c, k0, &full[s]);
          } else {
            tma_load_2d(sb, &maps.b, k0, I.n0, &full[s]);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: accumulator t & 1 of the two in tensor memory for the t-th item
      constexpr uint32_t idesc = sbp_umma::instr_desc_bf16_f32(BM, BN, A_MN, B_MN);
      int it = 0, t = 0;
      for (int w = blockIdx.x; w < items && !*(volatile int*)fail; w += gridDim.x, ++t) {
        const Item I = item(w, tm, tn, k_per, K, n_fast);
        const int nk = (I.ke - I.kb + BK - 1) / BK;
        const int buf = t & 1, ause = t >> 1;
        if (ause > 0 && !wait(&acc_empty[buf], (ause - 1) & 1)) {
          atomicOr(fail, 1);
          break;
        }
        fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(buf * ACC_COLS);
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = it % STAGES, use = it / STAGES;
          if (!wait(&full[s], use & 1)) {
            atomicOr(fail, 1);
            ok = false;
            break;
          }
          fence_after_sync();
          const uint32_t sa = sbp::smem_u32(base + s * STAGE_BYTES);
          const uint32_t sb = sa + A_BYTES;
#pragma unroll
          for (int k16 = 0; k16 < BK / 16; ++k16) {
            const uint64_t ad = A_MN ? sbp_umma::mnmajor_desc(sa, k16) : sbp_umma::kmajor_desc(sa, k16);
            const uint64_t bd = B_MN ? sbp_umma::mnmajor_desc(sb, k16) : sbp_umma::kmajor_desc(sb, k16);
            mma_bf16(acc, ad, bd, idesc, (kt > 0 || k16 > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);  // the accumulator is complete once every MMA above is
      }
      // before the tensor memory is freed, every MMA issued here has to have completed
      mma_commit(done);
      if (!wait(done, 0)) atomicOr(fail, 1);
    }
  } else {
    // epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31, i.e. those rows of the tile, and
    // the column chunks of its half of the tile
    const int lg = warp & 3;
    const int c0 = ((warp - 2) >> 2) * (BN / 64);
    unsigned char* wbuf = epi + (warp - 2) * EPI_WARP_BYTES;
    float* tile = reinterpret_cast<float*>(wbuf);
    const bool split = k_per < K;
    const bool tma = epi_mode != kEpiDirect;
    int t = 0, chunks_stored = 0;
    for (int w = blockIdx.x; w < items; w += gridDim.x, ++t) {
      const Item I = item(w, tm, tn, k_per, K, n_fast);
      const int buf = t & 1, use = t >> 1;
      const bool got = wait(&acc_full[buf], use & 1);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) atomicOr(fail, 1);
        break;
      }
      fence_after_sync();
      const uint32_t acc = tmem + (uint32_t)(buf * ACC_COLS) + ((uint32_t)(lg * 32) << 16);
      const int my_m = I.m0 + lg * 32 + lane;
      const float my_bias = (bias && I.kb == 0 && my_m < M) ? bias[my_m] : 0.f;
#pragma unroll 1
      for (int c = c0; c < c0 + BN / 64; ++c) {
        const int nb = I.n0 + 32 * c;
        if (nb >= N) break;  // uniform over the warp
        float v[32];
        tmem_ld32(acc + (uint32_t)(32 * c), v);
        if (tma) {
          // bias and ReLU in registers (this thread holds row my_m), then the 32 x 32 box into the
          // warp's buffer in the 128-byte swizzled layout the store map reads, and a TMA store (or
          // reduce-add) of the box; rows and columns beyond C are clipped by TMA
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            v[j] += my_bias;
            if (relu) v[j] = fmaxf(v[j], 0.f);
          }
          unsigned char* sb = wbuf;
          if (lane == 0 && chunks_stored >= 1)
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // the last store has read the buffer
          __syncwarp();
          if (epi_mode == kEpiTmaStoreBf16) {
            // BF16 rows of 64 bytes in the 64-byte swizzle (16-byte granule g of row r at
            // g ^ ((r / 2) % 4)), for a 32 x 32 BF16 box
            uint4* row = reinterpret_cast<uint4*>(sb + lane * 64);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              uint32_t w[4];
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const __nv_bfloat162 p = __floats2bfloat162_rn(v[8 * g + 2 * h], v[8 * g + 2 * h + 1]);
                w[h] = *reinterpret_cast<const uint32_t*>(&p);
              }
              row[g ^ ((lane >> 1) & 3)] = make_uint4(w[0], w[1], w[2], w[3]);
            }
          } else {
            float4* row = reinterpret_cast<float4*>(sb + lane * 128);
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4)
              row[j4 ^ (lane & 7)] = make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
          }
          sbp::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) tma_store_2d(&maps.c, nb, I.m0 + lg * 32, sb, epi_mode == kEpiTmaAdd);
          ++chunks_stored;
          continue;
        }
        // transpose through the warp's tile so that a store covers 32 consecutive columns (columns
        // rotated by the row: conflict-free writes of a row and reads of a column)
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[lane * 32 + ((j + lane) & 31)] = v[j];
        __syncwarp();
        const int n = nb + lane;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const int m = I.m0 + lg * 32 + r;
          if (m >= M) break;  // uniform over the warp
          float x = tile[r * 32 + ((lane + r) & 31)] + ((bias && I.kb == 0) ? bias[m] : 0.f);
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
      fence_before_sync();
      mbar_arrive(&acc_empty[buf]);  // this thread has read its part of the accumulator
    }
    // the stores read their buffers after this CTA's last instruction unless it waits for them
    if (lane == 0 && tma) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)fail) atomicOr(&g_tc_status, 1u);
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

// Encoded tensor maps, reused for repeated calls on the same operands (a network's GEMMs see
// the same buffers every iteration): a small table with round-robin replacement.
struct MapKey {
  const void* base;
  long long rows, cols, ld;
  int box_cols, box_rows, dev, fp32;
};
struct MapEntry {
  MapKey key;
  CUtensorMap map;
  bool used = false;
};
constexpr int kMapCache = 64;
std::mutex g_map_mutex;
MapEntry g_maps[kMapCache];
int g_map_next = 0;

bool encode_uncached(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld, int box_cols,
                     int box_rows, bool fp32);

// 2D tensor map of a row-major bf16 (or FP32) matrix with `rows` rows of `cols` elements (row
// pitch ld elements), box of box_cols x box_rows, zero fill outside the matrix; the swizzle spans
// one box row: 128 bytes (operand tiles, FP32 output boxes) or 64 bytes (BF16 output boxes).
bool encode(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld, int box_cols,
            int box_rows, bool fp32 = false) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  const MapKey k{base, rows, cols, ld, box_cols, box_rows, dev, fp32 ? 1 : 0};
  std::lock_guard<std::mutex> lock(g_map_mutex);
  for (auto& e : g_maps)
    if (e.used && e.key.base == k.base && e.key.rows == k.rows && e.key.cols == k.cols && e.key.ld == k.ld &&
        e.key.box_cols == k.box_cols && e.key.box_rows == k.box_rows && e.key.dev == k.dev && e.key.fp32 == k.fp32) {
      *m = e.map;
      return true;
    }
  if (!encode_uncached(m, base, rows, cols, ld, box_cols, box_rows, fp32)) return false;
  MapEntry& slot = g_maps[g_map_next];
  g_map_next = (g_map_next + 1) % kMapCache;
  slot.key = k;
  slot.map = *m;
  slot.used = true;
  return true;
}

bool encode_uncached(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld, int box_cols,
                     int box_rows, bool fp32) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  const int es_bytes = fp32 ? 4 : 2;
  const int row_bytes = box_cols * es_bytes;
  if (row_bytes != 128 && row_bytes != 64) return false;
  const CUtensorMapSwizzle swz = row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * es_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
             dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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
  const int tn = (N + BN - 1) / BN, tm = (M + BM - 1) / BM;
  int k_per = K;
  const long long tiles = (long long)tm * tn;
  // split K when the output tiles alone would leave SMs idle (FP32 output, plain sum)
  if (!c_bf16 && !relu && beta == 0.f && tiles < sms && K >= 8 * BK) {
    long long splits = (sms + tiles - 1) / tiles;
    splits = splits < K / (4 * BK) ? splits : K / (4 * BK);
    if (splits > 1) k_per = (int)(((K + splits - 1) / splits + BK - 1) / BK * BK);
  }
  const long long items = tiles * ((K + k_per - 1) / k_per);
  // TMA epilogue for outputs without accumulation (FP32: store, or reduce-add of split K; BF16:
  // store) when C suits TMA (16-byte aligned base, rows a multiple of 16 bytes); the direct path
  // otherwise
  int epi_mode = kEpiDirect;
  if (!c_bf16 && beta == 0.f && ldc % 4 == 0 && (uintptr_t)C % 16 == 0 &&
      encode(&maps.c, C, M, N, ldc, 32, 32, true))
    epi_mode = k_per < K ? kEpiTmaAdd : kEpiTmaStore;
  if (c_bf16 && beta == 0.f && k_per == K && ldc % 8 == 0 && (uintptr_t)C % 16 == 0 &&
      encode(&maps.c, C, M, N, ldc, 32, 32, false))
    epi_mode = kEpiTmaStoreBf16;
  if (items > (1LL << 30)) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  if (k_per < K) {
    e = ldc == N ? cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * N, st)
                 : cudaMemset2DAsync(C, sizeof(float) * (size_t)ldc, 0, sizeof(float) * (size_t)N, (size_t)M, st);
    if (e != cudaSuccess) return e;
  }
  // n tiles fastest when B fits in L2 with room to spare (a third of GB300's 126 MB)
  constexpr double kL2Bytes = 126.0e6;
  const int n_fast = (double)K * N * 2.0 <= kL2Bytes / 3.0 ? 1 : 0;
  // persistent: one CTA per SM (its shared memory and tensor memory fill the SM)
  const unsigned grid = (unsigned)(items < sms ? items : sms);
  // the shared-memory attribute belongs to the device: set once per device and kernel variant
  static std::mutex attr_mutex;
  static bool attr_set[64][4] = {};
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  auto launch = [&](auto kern, int variant) -> cudaError_t {
    {
      std::lock_guard<std::mutex> lock(attr_mutex);
      if (dev >= 64 || !attr_set[dev][variant]) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (r != cudaSuccess) return r;
        if (dev < 64) attr_set[dev][variant] = true;
      }
    }
    kern<<<grid, THREADS, SMEM_BYTES, st>>>(maps, M, N, K, k_per, tm, tn, (int)items, C, ldc, c_bf16, bias, relu,
                                           beta, epi_mode, n_fast);
    return cudaGetLastError();
  };
  const bool a_mn = ta != 0, b_mn = tb == 0;
  if (a_mn && b_mn) return launch(gemm_tc_kernel<true, true>, 3);
  if (a_mn) return launch(gemm_tc_kernel<true, false>, 2);
  if (b_mn) return launch(gemm_tc_kernel<false, true>, 1);
  return launch(gemm_tc_kernel<false, false>, 0);
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
