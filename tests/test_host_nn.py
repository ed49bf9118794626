"""The surrogate network's layout kernels on the CPU: tests/host_nn.cpp compiles the per-element
bodies of csrc/nn_elem.cuh (im2col, col2im, the moment combination and its backward) as host
C++.  Composed with plain matrix products (what the tensor-core GEMM computes) they give the
oracle network's direct-sum convolution and its input gradient, over ragged shapes, kernel
widths and paddings; the moment combination gives its definition, sum_c m_c G_c; the input's
Fourier features are x, then sin(2^k pi x), cos(2^k pi x) per input in the documented rows."""
import ctypes

import numpy as np
import pytest

from oracle.surrogate_net import conv1d, conv1d_backward, round_bf16

from host_build import build


@pytest.fixture(scope="module")
def hostnn(tmp_path_factory):
    so = build("host_nn.cpp", tmp_path_factory.mktemp("hostnn") / "libhostnn.so", shared=True)
    lib = ctypes.CDLL(so)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.host_conv_forward.argtypes = [P, P, P] + [I] * 6
    lib.host_conv_backward_dx.argtypes = [P, P, P] + [I] * 6
    lib.host_moment_combine.argtypes = [P] * 5 + [I] * 3
    lib.host_fourier_features.argtypes = [P, P] + [I] * 3
    return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


@pytest.mark.parametrize("C,B,T,Co", [(3, 2, 16, 4), (5, 3, 7, 2), (1, 1, 5, 3)])
def test_convolution_forward_and_input_gradient_match_oracle(hostnn, C, B, T, Co):
    import oracle.surrogate_net as sn
    kw, pad = sn.KW, sn.PAD
    rng = np.random.default_rng(C * 100 + T)
    x = _f32(rng.normal(size=(C, B, T)))
    W = _f32(rng.normal(size=(Co, C * kw)))
    y = np.zeros((Co, B, T), np.float32)
    hostnn.host_conv_forward(x.ctypes.data, W.ctypes.data, y.ctypes.data, C, B, T, Co, kw, pad)
    want = conv1d(round_bf16(x.astype(np.float64)), round_bf16(W.astype(np.float64)), np.zeros(Co))
    assert np.abs(y - want).max() < 1e-6 * max(1.0, np.abs(want).max())
    dy = _f32(rng.normal(size=(Co, B, T)))
    dx = np.zeros((C, B, T), np.float32)
    hostnn.host_conv_backward_dx(W.ctypes.data, dy.ctypes.data, dx.ctypes.data, C, B, T, Co, kw, pad)
    want_dx = conv1d_backward(x.astype(np.float64), W.astype(np.float64), dy.astype(np.float64))[0]
    assert np.abs(dx - want_dx).max() < 1e-5 * max(1.0, np.abs(want_dx).max())


@pytest.mark.parametrize("n_out,B,T", [(4, 3, 5), (1, 2, 7), (6, 1, 1)])
def test_moment_combination_and_backward(hostnn, n_out, B, T):
    rng = np.random.default_rng(n_out + 10 * T)
    G = _f32(rng.normal(size=(6, n_out, B, T)))
    m = _f32(rng.normal(size=(6, B)))
    dy = _f32(rng.normal(size=(n_out, B, T)))
    y = np.zeros((n_out, B, T), np.float32)
    dG = np.zeros((6, n_out, B, T), np.float32)
    hostnn.host_moment_combine(G.ctypes.data, m.ctypes.data, y.ctypes.data, dy.ctypes.data, dG.ctypes.data,
                               n_out, B, T)
    want = np.einsum("cb,cobt->obt", m.astype(np.float64), round_bf16(G.astype(np.float64)))
    assert np.abs(y - want).max() < 1e-5 * max(1.0, np.abs(want).max())
    want_dG = m[:, None, :, None].astype(np.float64) * round_bf16(dy.astype(np.float64))[None]
    assert np.abs(dG - round_bf16(want_dG)).max() <= 2.0 ** -8 * np.abs(want_dG).max()


@pytest.mark.parametrize("n_in,B,L", [(3, 5, 4), (1, 7, 1), (2, 3, 0), (3, 2, 6)])
def test_fourier_features(hostnn, n_in, B, L):
    rng = np.random.default_rng(n_in * 7 + L)
    x = _f32(rng.uniform(-1, 1, size=(n_in, B)))
    y = np.zeros((n_in * (1 + 2 * L), B), np.float32)
    hostnn.host_fourier_features(x.ctypes.data, y.ctypes.data, n_in, B, L)
    xd = x.astype(np.float64)
    rows = [xd[i] for i in range(n_in)]
    for i in range(n_in):
        for k in range(L):
            rows += [np.sin(2.0 ** k * np.pi * xd[i]), np.cos(2.0 ** k * np.pi * xd[i])]
    want = round_bf16(np.stack(rows))
    # BF16 rounding of FP32 sines: within one BF16 unit of the rounded FP64 value
    assert np.abs(y - want).max() <= 2.0 ** -7 * max(1.0, np.abs(want).max())
