// Per-element bodies of the surrogate network's layout kernels (nn.cu): im2col and col2im of
// the width-kw, zero-padded 1D convolution, and the moment combination of the output layer
// with its backward.  Element e of the kernels' flat output enumeration.  Device code of those
// kernels; without nvcc the same source compiles as host C++, so that the index arithmetic can
// be checked on a CPU.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

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

// y[o][b*T + t] = sum_c m[c][b] G[(c*n_out + o)][b*T + t]  (G BF16, y FP32)
__device__ __forceinline__ void moment_combine_at(const __nv_bfloat16* __restrict__ G, const float* __restrict__ m,
                                                  float* __restrict__ y, int n_out, int B, int T, long long e) {
  const int o = (int)(e / ((long long)B * T));
  const long long col = e % ((long long)B * T);
  const int b = (int)(col / T);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 6; ++c) s += m[c * B + b] * __bfloat162float(G[((long long)c * n_out + o) * B * T + col]);
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

// Fourier features of the network input: y[j][b] (BF16, [n_in (1 + 2 L)][B]) for x[i][b] (FP32,
// [n_in][B], normalised to [-1, 1]): rows 0..n_in-1 are x itself, then for each input i and
// k = 0..L-1 the pair sin(2^k pi x), cos(2^k pi x) (row n_in + 2 (i L + k) + 0 / 1).
__device__ __forceinline__ void fourier_features_at(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                                    int n_in, int B, int L, long long e) {
  const int j = (int)(e / B), b = (int)(e % B);
  float v;
  if (j < n_in) {
    v = x[(long long)j * B + b];
  } else {
    const int r = j - n_in;
    const int i = r / (2 * L), k = (r / 2) % L;
    const float a = 3.14159265358979f * ldexpf(x[(long long)i * B + b], k);
    v = (r & 1) ? cosf(a) : sinf(a);
  }
  y[e] = __float2bfloat16(v);
}

}  // namespace sbp_nn
