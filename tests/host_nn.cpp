// The surrogate network's layout kernels (im2col_at, col2im_at, moment_combine_at,
// moment_combine_bwd_at of paper_2011_02600_gb300/csrc/nn_elem.cuh) compiled as host C++, with
// the plain matrix products the tensor-core GEMM computes, for a width-kw convolution:
//   forward   Y = W . im2col(X)            (X, W rounded to BF16 as the library stores them)
//   backward  dX = col2im(W^T . dY)
// and the moment combination with its backward.  Built by tests/test_host_nn.py.
#include <vector>

#include "nn_elem.cuh"

using namespace sbp_nn;

// X [C][B*T], W [Co][C*kw] (FP32 in, rounded to BF16), Y [Co][B*T] (FP32, FP64 sums)
extern "C" void host_conv_forward(const float* X, const float* W, float* Y, int C, int B, int T, int Co, int kw,
                                  int pad) {
  const long long BT = (long long)B * T, R = (long long)C * kw;
  std::vector<__nv_bfloat16> xb(C * BT), xc(R * BT);
  for (long long i = 0; i < C * BT; ++i) xb[i] = __float2bfloat16(X[i]);
  for (long long e = 0; e < R * BT; ++e) im2col_at(xb.data(), xc.data(), B, T, kw, pad, e);
  for (int o = 0; o < Co; ++o)
    for (long long col = 0; col < BT; ++col) {
      double s = 0.0;
      for (long long r = 0; r < R; ++r)
        s += (double)__bfloat162float(__float2bfloat16(W[o * R + r])) * (double)__bfloat162float(xc[r * BT + col]);
      Y[o * BT + col] = (float)s;
    }
}

// dX [C][B*T] = col2im(W^T dY), W [Co][C*kw], dY [Co][B*T] (FP32)
extern "C" void host_conv_backward_dx(const float* W, const float* dY, float* dX, int C, int B, int T, int Co, int kw,
                                      int pad) {
  const long long BT = (long long)B * T, R = (long long)C * kw;
  std::vector<float> dxc(R * BT);
  for (long long r = 0; r < R; ++r)
    for (long long col = 0; col < BT; ++col) {
      double s = 0.0;
      for (int o = 0; o < Co; ++o) s += (double)W[o * R + r] * (double)dY[o * BT + col];
      dxc[r * BT + col] = (float)s;
    }
  for (long long e = 0; e < C * BT; ++e) col2im_at(dxc.data(), dX, B, T, kw, pad, e);
}

// y [n_out][B*T] from G [6*n_out][B*T] (rounded to BF16) and m [6][B]; dG [6*n_out][B*T] (BF16,
// returned as FP32) from dy
extern "C" void host_moment_combine(const float* G, const float* m, float* y, const float* dy, float* dG, int n_out,
                                    int B, int T) {
  const long long BT = (long long)B * T;
  std::vector<__nv_bfloat16> gb(6 * n_out * BT);
  for (long long i = 0; i < 6 * n_out * BT; ++i) gb[i] = __float2bfloat16(G[i]);
  for (long long e = 0; e < n_out * BT; ++e) moment_combine_at(gb.data(), m, y, n_out, B, T, e);
  std::vector<__nv_bfloat16> dyb(n_out * BT), dgb(6 * n_out * BT);
  for (long long i = 0; i < n_out * BT; ++i) dyb[i] = __float2bfloat16(dy[i]);
  for (long long e = 0; e < 6 * n_out * BT; ++e) moment_combine_bwd_at(dyb.data(), m, dgb.data(), n_out, B, T, e);
  for (long long i = 0; i < 6 * n_out * BT; ++i) dG[i] = __bfloat162float(dgb[i]);
}

// y [n_in (1 + 2 L)][B] (BF16, returned as FP32): the Fourier features of x [n_in][B]
extern "C" void host_fourier_features(const float* x, float* y, int n_in, int B, int L) {
  const long long n = (long long)n_in * (1 + 2 * L) * B;
  std::vector<__nv_bfloat16> yb(n);
  for (long long e = 0; e < n; ++e) fourier_features_at(x, yb.data(), n_in, B, L, e);
  for (long long e = 0; e < n; ++e) y[e] = __bfloat162float(yb[e]);
}
