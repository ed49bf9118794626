// Kernels of the learned surrogate: BF16 tensor-core GEMMs with FP32
// accumulation and the small layer kernels around it (1D convolution as
// im2col + GEMM, nearest upsampling, ReLU, bias gradients, MSE loss, Adam).
// sbp_nn_gemm runs the tcgen05 kernel of nn_tc.cu where the operands allow it;
// the mma.sync kernels below serve small and unaligned products.
//
// Matrices are row-major.  The GEMM computes
//     C[M x N] = beta * C + op(A)[M x K] op(B)[K x N] (+ bias[m]) (ReLU)
// with op(A) = A (stored M x K) or A^T (stored K x M), op(B) = B (stored K x N) or
// B^T (stored N x K).  A 128 x 128 block tile, 32-deep K steps, 8 warps of 64 x 32;
// tiles are staged in shared memory as A[m][k] and B^T[n][k] and fed to
// mma.sync.m16n8k16 (BF16 in, FP32 accumulate) through ldmatrix.
#include <cuda_bf16.h>
#include <algorithm>
#include <mutex>
#include <stdint.h>

#include "nn_elem.cuh"
#include "sbp.h"

namespace sbp_nn {

constexpr int BM = 128, BN = 128, BK = 32, PAD = 8;
constexpr int LDS = BK + PAD;  // shared row stride (bf16 elements)

__device__ __forceinline__ unsigned s_addr(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s_addr(p)));
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                        long long lda, int ta, const __nv_bfloat16* __restrict__ B,
                                                        long long ldb, int tb, void* C, long long ldc, int c_bf16,
                                                        const float* __restrict__ bias, int relu, float beta) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][LDS];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][LDS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 2) * 64;  // 2 x 4 warps: 64 (m) x 32 (n) each
  const int wn = (warp & 3) * 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);

  for (int k0 = 0; k0 < K; k0 += BK) {
    // stage op(A)[m0.., k0..] as As[m][k] and op(B)[k0.., n0..] as Bs[n][k]
    for (int e = tid; e < BM * BK; e += 256) {
      int m, k;
      if (ta) {  // stored K x M: walk m fastest (coalesced)
        m = e % BM;
        k = e / BM;
      } else {
        k = e % BK;
        m = e / BK;
      }
      const int gm = m0 + m, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gm < M && gk < K) v = ta ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[m][k] = v;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int n, k;
      if (tb) {  // stored N x K: walk k fastest
        k = e % BK;
        n = e / BK;
      } else {
        n = e % BN;
        k = e / BN;
      }
      const int gn = n0 + n, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gn < N && gk < K) v = tb ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[n][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[4][4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int r = wm + mi * 16 + (lane & 15);
        const int c = kk + (lane >> 4) * 8;
        ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], &As[r][c]);
      }
      unsigned bf[4][2];
#pragma unroll
      for (int nj = 0; nj < 4; nj += 2) {
        // two n8 tiles at once: lanes 0-7 rows n..n+7 k, 8-15 k+8, 16-23 rows n+8.. k, 24-31 k+8
        const int r = wn + nj * 8 + (lane & 7) + ((lane >> 4) << 3);
        const int c = kk + ((lane >> 3) & 1) * 8;
        unsigned r0, r1, r2, r3;
        ldsm_x4(r0, r1, r2, r3, &Bs[r][c]);
        bf[nj][0] = r0;
        bf[nj][1] = r1;
        bf[nj + 1][0] = r2;
        bf[nj + 1][1] = r3;
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) mma_bf16(acc[mi][nj], af[mi], bf[nj][0], bf[nj][1]);
    }
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int nj = 0; nj < 4; ++nj)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gm = m0 + wm + mi * 16 + (lane >> 2) + h * 8;
        if (gm >= M) continue;
        const float bv = bias ? bias[gm] : 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int gn = n0 + wn + nj * 8 + (lane & 3) * 2 + q;
          if (gn >= N) continue;
          float v = acc[mi][nj][h * 2 + q] + bv;
          const long long idx = (long long)gm * ldc + gn;
          if (c_bf16) {
            if (relu) v = fmaxf(v, 0.f);
            ((__nv_bfloat16*)C)[idx] = __float2bfloat16(v);
          } else {
            if (beta != 0.f) v += beta * ((float*)C)[idx];
            if (relu) v = fmaxf(v, 0.f);
            ((float*)C)[idx] = v;
          }
        }
      }
}

// ---------------------------------------------------------------------------------------------
// Pipelined GEMM for operands whose leading dimensions are multiples of 8 (16-byte rows):
// each operand tile is copied with 16-byte cp.async vectors along the operand's contiguous
// dimension into a three-stage shared-memory ring, keeping that orientation: "K-major" tiles
// [row][k] when k is contiguous (A stored M x K, or B stored N x K) and "MN-major" tiles
// [k][row] otherwise; ldmatrix (K-major) or ldmatrix.trans (MN-major) produces the same
// mma.sync fragments either way.  Vectors past M, N or K are zero-filled by the copy.
// Split-K (blockIdx.z over K ranges) adds partial tiles atomically into an FP32 output that
// the host zeroed; it is used only without accumulation, ReLU or BF16 output.
constexpr int PBM = 128, PBN = 128, PBK = 64, PSTAGES = 3;
constexpr int KM_LD = PBK + 8;  // K-major tile row stride (bf16 elements)
constexpr int MN_LD = PBM + 8;  // MN-major tile row stride
constexpr int PTILE = PBM * KM_LD > PBK * MN_LD ? PBM * KM_LD : PBK * MN_LD;
constexpr int PSMEM = PSTAGES * 2 * PTILE * 2;  // bytes

__device__ __forceinline__ void ldsm_x4_t(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s_addr(p)));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s_addr(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Copy the 128 x PBK tile of an operand whose rows (m or n) start at r0 and k at k0 into t.
//   kmajor: stored [R][ld] with k contiguous -> t[row][k];  else stored [K][ld] -> t[k][row].
__device__ __forceinline__ void load_tile(__nv_bfloat16* t, const __nv_bfloat16* __restrict__ X, long long ld,
                                          bool kmajor, int R, int K, int r0, int k0, int tid) {
  constexpr int VR = PBK / 8;  // 16-byte vectors per K-major row
#pragma unroll
  for (int i = 0; i < PBM * PBK / 8 / 256; ++i) {
    const int v = tid + i * 256;
    int r, k, valid;
    const __nv_bfloat16* src;
    __nv_bfloat16* dst;
    if (kmajor) {
      r = v / VR;
      k = (v % VR) * 8;
      const int gr = r0 + r, gk = k0 + k;
      valid = gr < R ? max(0, min(8, K - gk)) : 0;
      src = valid ? X + (long long)gr * ld + gk : X;
      dst = t + r * KM_LD + k;
    } else {
      k = v >> 4;
      r = (v & 15) * 8;
      const int gr = r0 + r, gk = k0 + k;
      valid = gk < K ? max(0, min(8, R - gr)) : 0;
      src = valid ? X + (long long)gk * ld + gr : X;
      dst = t + k * MN_LD + r;
    }
    cp_async16(dst, src, valid * 2);
  }
}

__global__ void __launch_bounds__(256) gemm_bf16_pipe_kernel(int M, int N, int K, int k_per,
                                                             const __nv_bfloat16* __restrict__ A, long long lda,
                                                             int ta, const __nv_bfloat16* __restrict__ B,
                                                             long long ldb, int tb, void* C, long long ldc,
                                                             int c_bf16, const float* __restrict__ bias, int relu,
                                                             float beta) {
  extern __shared__ __align__(16) unsigned char nn_smem[];
  __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(nn_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 2) * 64;  // 2 x 4 warps: 64 (m) x 32 (n) each
  const int wn = (warp & 3) * 32;
  const int m0 = blockIdx.y * PBM, n0 = blockIdx.x * PBN;
  const int kb = blockIdx.z * k_per, ke = min(K, kb + k_per);
  const bool akm = !ta, bkm = tb;  // K-major tiles
  const int nt = (ke - kb + PBK - 1) / PBK;
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  auto As = [&](int st) { return sm + (2 * st) * PTILE; };
  auto Bs = [&](int st) { return sm + (2 * st + 1) * PTILE; };
#pragma unroll
  for (int st = 0; st < PSTAGES - 1; ++st) {
    if (st < nt) {
      load_tile(As(st), A, lda, akm, M, ke, m0, kb + st * PBK, tid);
      load_tile(Bs(st), B, ldb, bkm, N, ke, n0, kb + st * PBK, tid);
    }
    cp_async_commit();
  }
  for (int t = 0; t < nt; ++t) {
    cp_async_wait1();
    __syncthreads();
    {
      const int tn = t + PSTAGES - 1;
      if (tn < nt) {
        load_tile(As(tn % PSTAGES), A, lda, akm, M, ke, m0, kb + tn * PBK, tid);
        load_tile(Bs(tn % PSTAGES), B, ldb, bkm, N, ke, n0, kb + tn * PBK, tid);
      }
      cp_async_commit();
    }
    const __nv_bfloat16* as = As(t % PSTAGES);
    const __nv_bfloat16* bs = Bs(t % PSTAGES);
#pragma unroll
    for (int kk = 0; kk < PBK; kk += 16) {
      unsigned af[4][4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        if (akm) {
          ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3],
                  as + (wm + mi * 16 + (lane & 15)) * KM_LD + kk + (lane >> 4) * 8);
        } else {
          const int q = lane >> 3, r = lane & 7;
          ldsm_x4_t(af[mi][0], af[mi][1], af[mi][2], af[mi][3],
                    as + (kk + (q >> 1) * 8 + r) * MN_LD + wm + mi * 16 + (q & 1) * 8);
        }
      }
      unsigned bf[4][2];
#pragma unroll
      for (int nj = 0; nj < 4; nj += 2) {
        unsigned r0, r1, r2, r3;
        if (bkm) {
          const int r = wn + nj * 8 + (lane & 7) + ((lane >> 4) << 3);
          const int c = kk + ((lane >> 3) & 1) * 8;
          ldsm_x4(r0, r1, r2, r3, bs + r * KM_LD + c);
        } else {
          const int q = lane >> 3, r = lane & 7;
          ldsm_x4_t(r0, r1, r2, r3, bs + (kk + (q & 1) * 8 + r) * MN_LD + wn + nj * 8 + (q >> 1) * 8);
        }
        bf[nj][0] = r0;
        bf[nj][1] = r1;
        bf[nj + 1][0] = r2;
        bf[nj + 1][1] = r3;
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) mma_bf16(acc[mi][nj], af[mi], bf[nj][0], bf[nj][1]);
    }
  }
  cp_async_wait1();
  const bool split = gridDim.z > 1;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int nj = 0; nj < 4; ++nj)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gm = m0 + wm + mi * 16 + (lane >> 2) + h * 8;
        if (gm >= M) continue;
        const float bv = (bias && blockIdx.z == 0) ? bias[gm] : 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int gn = n0 + wn + nj * 8 + (lane & 3) * 2 + q;
          if (gn >= N) continue;
          float v = acc[mi][nj][h * 2 + q] + bv;
          const long long idx = (long long)gm * ldc + gn;
          if (split) {
            atomicAdd((float*)C + idx, v);
          } else if (c_bf16) {
            if (relu) v = fmaxf(v, 0.f);
            ((__nv_bfloat16*)C)[idx] = __float2bfloat16(v);
          } else {
            if (beta != 0.f) v += beta * ((float*)C)[idx];
            if (relu) v = fmaxf(v, 0.f);
            ((float*)C)[idx] = v;
          }
        }
      }
}

// im2col of a 1D convolution (kernel width kw, zero padding pad): X [C][B*T] ->
// Xc [(c*kw + k)][b*T + t] = X[c][b*T + t + k - pad] (zero outside 0..T-1).
__global__ void im2col_kernel(const __nv_bfloat16* __restrict__ X, __nv_bfloat16* __restrict__ Xc, int C, int B,
                              int T, int kw, int pad) {
  const long long n = (long long)C * kw * B * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    im2col_at(X, Xc, B, T, kw, pad, e);
  }
}

// col2im: dX[c][b*T + t] = sum_k dXc[(c*kw + k)][b*T + t - k + pad]  (FP32)
__global__ void col2im_kernel(const float* __restrict__ dXc, float* __restrict__ dX, int C, int B, int T,
                              int kw, int pad) {
  const long long n = (long long)C * B * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    col2im_at(dXc, dX, B, T, kw, pad, e);
  }
}

// nearest upsampling x2 along time: [C][B*T] -> [C][B*2T]; backward sums pairs.
__global__ void upsample2_kernel(const __nv_bfloat16* __restrict__ X, __nv_bfloat16* __restrict__ Y, long long rows,
                                 int T) {
  const long long n = rows * 2 * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / (2 * T);
    const int t2 = (int)(e % (2 * T));
    Y[e] = X[r * T + t2 / 2];
  }
}

__global__ void upsample2_bwd_kernel(const float* __restrict__ dY, float* __restrict__ dX, long long rows, int T) {
  const long long n = rows * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / T;
    const int t = (int)(e % T);
    dX[e] = dY[r * 2 * T + 2 * t] + dY[r * 2 * T + 2 * t + 1];
  }
}

// dZ = dA * (A > 0) for A = ReLU(Z): FP32 gradient in, BF16 out
__global__ void relu_bwd_kernel(const float* __restrict__ dA, const __nv_bfloat16* __restrict__ A,
                                __nv_bfloat16* __restrict__ dZ, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dZ[e] = __float2bfloat16(__bfloat162float(A[e]) > 0.f ? dA[e] : 0.f);
}

// db[m] = sum_n dZ[m][n]  (one block per row, fixed order)
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ dZ, float* __restrict__ db, int M, long long N) {
  __shared__ float red[256];
  const int m = blockIdx.x;
  float s = 0.f;
  for (long long n = threadIdx.x; n < N; n += blockDim.x) s += __bfloat162float(dZ[(long long)m * N + n]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[m] = red[0];
}

// mean squared error over n values: per-block FP64 partial sums of (y - t)^2 and dY = 2 (y - t) / n (BF16)
__global__ void mse_kernel(const float* __restrict__ Y, const float* __restrict__ Tg, __nv_bfloat16* __restrict__ dY,
                           long long n, double* __restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  const float sc = 2.f / (float)n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float d = Y[e] - Tg[e];
    s += (double)d * d;
    if (dY) dY[e] = __float2bfloat16(sc * d);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Adam on FP32 master weights; writes the BF16 copy used by the GEMMs.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ wb, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float wi = w[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[e] = wi;
    if (wb) wb[e] = __float2bfloat16(wi);
  }
}

// [F = C*T0][B] (feature-major MLP output) <-> [C][B*T0] (convolution layout), BF16
__global__ void mlp_to_conv_kernel(const __nv_bfloat16* __restrict__ H, __nv_bfloat16* __restrict__ X, int C, int T0,
                                   int B, int backward) {
  const long long n = (long long)C * T0 * B;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / ((long long)B * T0));
    const long long col = e % ((long long)B * T0);
    const int b = (int)(col / T0), t = (int)(col % T0);
    const long long h = ((long long)c * T0 + t) * B + b;
    if (backward)
      ((__nv_bfloat16*)H)[h] = X[e];
    else
      X[e] = H[h];
  }
}

// Moment combination: y[o][b*T + t] = sum_c m[c][b] G[(c*n_out + o)][b*T + t] (G FP32);
// backward: dG[(c*n_out + o)][b*T + t] = m[c][b] dy[o][b*T + t] (BF16).
__global__ void moment_combine_kernel(const __nv_bfloat16* __restrict__ G, const float* __restrict__ m, float* __restrict__ y,
                                      int n_out, int B, int T) {
  const long long n = (long long)n_out * B * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    moment_combine_at(G, m, y, n_out, B, T, e);
  }
}

__global__ void moment_combine_bwd_kernel(const __nv_bfloat16* __restrict__ dy, const float* __restrict__ m,
                                          __nv_bfloat16* __restrict__ dG, int n_out, int B, int T) {
  const long long n = 6LL * n_out * B * T;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    moment_combine_bwd_at(dy, m, dG, n_out, B, T, e);
  }
}

__global__ void fourier_features_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int n_in, int B,
                                        int L, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    fourier_features_at(x, y, n_in, B, L, e);
}

__global__ void cast_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = __float2bfloat16(x[e]);
}

inline unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace sbp_nn

namespace sbp {
void set_last_error(const char* msg);
}

namespace sbp_nn {
// nn_tc.cu: the tcgen05 GEMM (cudaErrorNotSupported when the operands do not suit TMA) and
// its status word.
cudaError_t launch_gemm_tc(int M, int N, int K, const void* A, long long lda, int ta, const void* B, long long ldb,
                           int tb, void* C, long long ldc, int c_bf16, const float* bias, int relu, float beta,
                           int sms, cudaStream_t st);
cudaError_t gemm_tc_status(unsigned* bits);
}  // namespace sbp_nn

namespace {
int nn_status(cudaError_t e) {
  if (e == cudaSuccess) return SBP_OK;
  sbp::set_last_error(cudaGetErrorString(e));
  return SBP_ERR_CUDA;
}
int nn_bad(const char* msg) {
  sbp::set_last_error(msg);
  return SBP_ERR_ARG;
}
// GEMM path (sbp_nn_set_gemm_path): 0 automatic, 1 mma.sync kernels only, 2 tcgen05 whenever possible.
int g_gemm_path = 0;

// SM count of the current device (152 on GB300, also the value taken if the query fails).
int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n <= 0)
    return 152;
  return n;
}
}  // namespace

using namespace sbp_nn;

extern "C" {

int sbp_nn_gemm(int32_t M, int32_t N, int32_t K, const void* A, int64_t lda, int32_t transA, const void* B,
                int64_t ldb, int32_t transB, void* C, int64_t ldc, int32_t c_bf16, const float* bias, int32_t relu,
                float beta, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0) return nn_bad("GEMM sizes must be positive");
  if (!A || !B || !C) return nn_bad("null GEMM operand");
  if (lda < (transA ? M : K) || ldb < (transB ? K : N) || ldc < N) return nn_bad("leading dimension too small");
  if (c_bf16 && beta != 0.f) return nn_bad("accumulation (beta) needs an FP32 output");
  const cudaStream_t st = (cudaStream_t)stream;
  const bool aligned = lda % 8 == 0 && ldb % 8 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0;
  // the tensor-core (tcgen05) kernel: TMA-loadable operands; automatically for tiles of at least
  // 128 x 128 (smaller products leave most of its 128 x 256 tile empty)
  const bool use_tc = aligned && g_gemm_path != 1 && (g_gemm_path == 2 || (M >= 128 && N >= 128 && K >= 64));
  if (use_tc) {
    cudaError_t e = launch_gemm_tc(M, N, K, A, lda, transA, B, ldb, transB, C, ldc, c_bf16, bias, relu, beta,
                                   device_sms(), st);
    if (e != cudaErrorNotSupported) return nn_status(e);
  }
  if (!aligned) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    if (grid.y > 65535) return nn_bad("M too large");
    gemm_bf16_kernel<<<grid, 256, 0, st>>>(M, N, K, (const __nv_bfloat16*)A, lda, transA, (const __nv_bfloat16*)B,
                                           ldb, transB, C, ldc, c_bf16, bias, relu, beta);
    return nn_status(cudaGetLastError());
  }
  dim3 grid((N + PBN - 1) / PBN, (M + PBM - 1) / PBM, 1);
  if (grid.y > 65535) return nn_bad("M too large");
  // split K when the output tiles alone would leave most SMs idle (FP32 output, plain sum);
  // the target is two resident CTAs per SM
  int k_per = K;
  const long long tiles = (long long)grid.x * grid.y;
  const long long slots = 2LL * device_sms();
  if (!c_bf16 && !relu && beta == 0.f && tiles < slots && K >= 8 * PBK) {
    long long splits = (slots + tiles - 1) / tiles;
    splits = std::min<long long>(splits, K / (4 * PBK));
    if (splits > 1) {
      k_per = (int)(((K + splits - 1) / splits + PBK - 1) / PBK * PBK);
      grid.z = (unsigned)((K + k_per - 1) / k_per);
    }
  }
  cudaError_t e = cudaSuccess;
  if (grid.z > 1) {
    e = ldc == N ? cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * N, st)
                 : cudaMemset2DAsync(C, sizeof(float) * (size_t)ldc, 0, sizeof(float) * (size_t)N, (size_t)M, st);
    if (e != cudaSuccess) return nn_status(e);
  }
  // the attribute belongs to the device: set once per device
  {
    static std::mutex m;
    static bool set[64] = {};
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nn_status(e);
    std::lock_guard<std::mutex> lock(m);
    if (dev >= 64 || !set[dev]) {
      e = cudaFuncSetAttribute(gemm_bf16_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PSMEM);
      if (e != cudaSuccess) return nn_status(e);
      if (dev < 64) set[dev] = true;
    }
  }
  gemm_bf16_pipe_kernel<<<grid, 256, PSMEM, st>>>(M, N, K, k_per, (const __nv_bfloat16*)A, lda, transA,
                                                  (const __nv_bfloat16*)B, ldb, transB, C, ldc, c_bf16, bias, relu,
                                                  beta);
  return nn_status(cudaGetLastError());
}

int sbp_nn_set_gemm_path(int32_t path) {
  if (path < 0 || path > 2) return nn_bad("GEMM path must be 0 (automatic), 1 (mma.sync) or 2 (tcgen05)");
  g_gemm_path = path;
  return SBP_OK;
}

int sbp_nn_status(uint32_t* bits) {
  if (!bits) return nn_bad("null output");
  unsigned v = 0;
  cudaError_t e = gemm_tc_status(&v);
  if (e != cudaSuccess) return nn_status(e);
  *bits = v;
  return SBP_OK;
}

int sbp_nn_im2col(const void* X, void* Xc, int32_t C, int32_t B, int32_t T, int32_t kw, int32_t pad, void* stream) {
  if (!X || !Xc || C <= 0 || B <= 0 || T <= 0 || kw <= 0 || pad < 0) return nn_bad("bad im2col arguments");
  const long long n = (long long)C * kw * B * T;
  im2col_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)X, (__nv_bfloat16*)Xc, C, B, T,
                                                                kw, pad);
  return nn_status(cudaGetLastError());
}

int sbp_nn_col2im(const float* dXc, void* dX, int32_t C, int32_t B, int32_t T, int32_t kw, int32_t pad,
                  void* stream) {
  if (!dXc || !dX || C <= 0 || B <= 0 || T <= 0 || kw <= 0 || pad < 0) return nn_bad("bad col2im arguments");
  const long long n = (long long)C * B * T;
  col2im_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(dXc, (float*)dX, C, B, T, kw, pad);
  return nn_status(cudaGetLastError());
}

int sbp_nn_upsample2(const void* X, void* Y, int64_t rows, int32_t T, int32_t backward, void* stream) {
  if (!X || !Y || rows <= 0 || T <= 0) return nn_bad("bad upsample arguments");
  if (backward)
    upsample2_bwd_kernel<<<grid_for(rows * T), 256, 0, (cudaStream_t)stream>>>((const float*)X, (float*)Y, rows, T);
  else
    upsample2_kernel<<<grid_for(rows * 2 * T), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)X,
                                                                                (__nv_bfloat16*)Y, rows, T);
  return nn_status(cudaGetLastError());
}

int sbp_nn_relu_backward(const float* dA, const void* A, void* dZ, int64_t n, void* stream) {
  if (!dA || !A || !dZ || n <= 0) return nn_bad("bad relu_backward arguments");
  relu_bwd_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(dA, (const __nv_bfloat16*)A, (__nv_bfloat16*)dZ, n);
  return nn_status(cudaGetLastError());
}

int sbp_nn_bias_grad(const void* dZ, float* db, int32_t M, int64_t N, void* stream) {
  if (!dZ || !db || M <= 0 || N <= 0) return nn_bad("bad bias_grad arguments");
  bias_grad_kernel<<<M, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)dZ, db, M, N);
  return nn_status(cudaGetLastError());
}

int sbp_nn_mse(const float* Y, const float* Tg, void* dY, int64_t n, double* partial, int32_t nblocks,
               void* stream) {
  if (!Y || !Tg || !partial || n <= 0 || nblocks <= 0) return nn_bad("bad mse arguments");
  mse_kernel<<<nblocks, 256, 0, (cudaStream_t)stream>>>(Y, Tg, (__nv_bfloat16*)dY, n, partial);
  return nn_status(cudaGetLastError());
}

int sbp_nn_adam(float* w, const float* g, float* m, float* v, void* w_bf16, int64_t n, float lr, float b1, float b2,
                float eps, int32_t step, void* stream) {
  if (!w || !g || !m || !v || n <= 0 || step < 1) return nn_bad("bad adam arguments");
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, (__nv_bfloat16*)w_bf16, n, lr, b1, b2, eps,
                                                              c1, c2);
  return nn_status(cudaGetLastError());
}

int sbp_nn_mlp_to_conv(void* H, void* X, int32_t C, int32_t T0, int32_t B, int32_t backward, void* stream) {
  if (!H || !X || C <= 0 || T0 <= 0 || B <= 0) return nn_bad("bad reshape arguments");
  mlp_to_conv_kernel<<<grid_for((long long)C * T0 * B), 256, 0, (cudaStream_t)stream>>>(
      (const __nv_bfloat16*)H, (__nv_bfloat16*)X, C, T0, B, backward);
  return nn_status(cudaGetLastError());
}

int sbp_nn_moment_combine(const void* G, const float* m, float* y, const void* dy, void* dG, int32_t n_out,
                          int32_t B, int32_t T, int32_t backward, void* stream) {
  if (!m || n_out <= 0 || B <= 0 || T <= 0) return nn_bad("bad moment_combine arguments");
  if (backward) {
    if (!dy || !dG) return nn_bad("moment_combine backward needs dy and dG");
    moment_combine_bwd_kernel<<<grid_for(6LL * n_out * B * T), 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)dy, m, (__nv_bfloat16*)dG, n_out, B, T);
  } else {
    if (!G || !y) return nn_bad("moment_combine needs G and y");
    moment_combine_kernel<<<grid_for((long long)n_out * B * T), 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16*)G, m, y, n_out, B, T);
  }
  return nn_status(cudaGetLastError());
}

int sbp_nn_fourier_features(const float* x, void* y, int32_t n_in, int64_t B, int32_t L, void* stream) {
  if (!x || !y || n_in <= 0 || B <= 0 || L < 0 || L > 16) return nn_bad("bad Fourier feature arguments");
  const long long n = (long long)n_in * (1 + 2 * L) * B;
  fourier_features_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, (__nv_bfloat16*)y, n_in, (int)B, L, n);
  return nn_status(cudaGetLastError());
}

int sbp_nn_cast_bf16(const float* x, void* y, int64_t n, void* stream) {
  if (!x || !y || n <= 0) return nn_bad("bad cast arguments");
  cast_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, (__nv_bfloat16*)y, n);
  return nn_status(cudaGetLastError());
}

}  // extern "C"
