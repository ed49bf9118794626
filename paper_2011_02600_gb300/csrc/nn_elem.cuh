// Per-element bodies of the surrogate network's layout kernels (nn.cu): im2col and col2im of
// the width-kw, zero-padded 1D convolution, and the moment combination of the output layer
// with its backward.  Element e of the kernels' flat output enumeration.  Device code of those
// kernels; without nvcc the same source compiles as host C++, so that the index arithmetic can
// be checked on a CPU.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sbp_nn {

// Xc [(c*kw + k)][b*T + t] = X[c][b*T + t + k - pad] (zero outside 0..T-1)
__device__ __forceinline__ void im2col_at(const __nv_bfloat16* __restrict__ X, __nv_bfloat16* __restrict__ Xc, int B,
                                          int T, int kw, int pad, long long e) {
  const long long col = e % ((long long)B * T);
  const long long row = e / ((long long)B * T);
  const int c = (int)(row / kw), k = (int)(row % kw);
  const int b = (int)(col / T), t = (int)(col % T);
  const int ts = t + k - pad;
  Xc[e] = (ts >= 0 && ts < T) ? X[(long long)c * B * T + (long long)b * T + ts] : __float2bfloat16(0.f);
}

// dX[c][b*T + t] = sum_k dXc[(c*kw + k)][b*T + t - k + pad]  (FP32)
__device__ __forceinline__ void col2im_at(const float* __restrict__ dXc, float* __restrict__ dX, int B, int T, int kw,
                                          int pad, long long e) {
  const int c = (int)(e / ((long long)B * T));
  const long long col = e % ((long long)B * T);
  const int b = (int)(col / T), t = (int)(col % T);
  float s = 0.f;
  for (int k = 0; k < kw; ++k) {
    const int tt = t - k + pad;
    if (tt >= 0 && tt < T) s += dXc[((long long)c * kw + k) * B * T + (long long)b * T + tt];
  }
  dX[e] = s;
}

// y[o][b*T + t] = sum_c m[c][b] G[(c*n_out + o)][b*T + t]  (G FP32)
__device__ __forceinline__ void moment_combine_at(const float* __restrict__ G, const float* __restrict__ m,
                                                  float* __restrict__ y, int n_out, int B, int T, long long e) {
  const int o = (int)(e / ((long long)B * T));
  const long long col = e % ((long long)B * T);
  const int b = (int)(col / T);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 6; ++c) s += m[c * B + b] * G[((long long)c * n_out + o) * B * T + col];
  y[e] = s;
}

// dG[(c*n_out + o)][b*T + t] = m[c][b] dy[o][b*T + t]  (BF16)
__device__ __forceinline__ void moment_combine_bwd_at(const __nv_bfloat16* __restrict__ dy, const float* __restrict__ m,
                                                      __nv_bfloat16* __restrict__ dG, int n_out, int B, int T,
                                                      long long e) {
  const long long row = e / ((long long)B * T);
  const long long col = e % ((long long)B * T);
  const int c = (int)(row / n_out), o = (int)(row % n_out);
  const int b = (int)(col / T);
  dG[e] = __float2bfloat16(m[c * B + b] * __bfloat162float(dy[(long long)o * B * T + col]));
}

}  // namespace sbp_nn
