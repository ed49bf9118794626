"""The learned surrogate's kernels and training.

* The BF16 tensor-core GEMM against numpy on the same BF16-rounded operands (FP32
  accumulation: 1e-5 relative; BF16 output: one BF16 rounding, 1e-2).
* Forward output and every weight/bias gradient of a small instance of the network
  against the oracle network (oracle/surrogate_net.py) on the same BF16 weights and
  inputs, with the oracle rounding to BF16 where the library stores BF16: what is left
  is FP32 against FP64 accumulation and the rare BF16 rounding it flips, 5e-3 relative
  (L2 over each tensor).  Against the all-FP64 oracle the BF16 storage itself shows:
  2^-9 relative per rounding, compounded over the ~12 layers between dL/dy and the
  first layer's gradient, bounded here by 1e-1.
* End to end on a reduced solver configuration: data from the batched solver, training
  by the library's kernels, held-out error against the solver, and the speed-up.
"""
import dataclasses

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _bf(x):
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(37, 61, 19), (128, 256, 320), (300, 70, 33), (192, 1024, 320), (7, 5, 300),
                                   (136, 200, 96), (40, 64, 1000), (264, 136, 64), (128, 640, 32768)])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_tensor_cores_vs_numpy(M, N, K, ta, tb):
    """Both GEMM kernels: the scalar-staged one (a leading dimension not a multiple of 8) and
    the pipelined one (ragged M, N, K edges; split K for the 128 x 640 x 32768 FP32 case)."""
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    rng = np.random.default_rng(M * 7 + N * 3 + K + ta * 5 + tb)
    A = _bf(rng.normal(size=(K, M) if ta else (M, K)))
    B = _bf(rng.normal(size=(N, K) if tb else (K, N)))
    bias = torch.as_tensor(rng.normal(size=M), dtype=torch.float32)
    An = A.float().numpy().astype(np.float64)
    Bn = B.float().numpy().astype(np.float64)
    ref = (An.T if ta else An) @ (Bn.T if tb else Bn) + bias.numpy()[:, None]
    Ad, Bd, bd = A.cuda(), B.cuda(), bias.cuda()
    lda, ldb = A.shape[1], B.shape[1]
    C = torch.empty(M, N, device="cuda")
    L.sbp_nn_gemm(M, N, K, Ad, lda, ta, Bd, ldb, tb, C, N, 0, bd, 0, 0.0, _stream())
    got = C.cpu().numpy()
    # FP32 accumulation: the rounding error of a K-term sum of random-sign terms grows like sqrt(K)
    tol = 1e-5 * max(1.0, (K / 1024) ** 0.5)
    assert np.abs(got - ref).max() < tol * np.abs(ref).max()
    # accumulate (beta = 1) and ReLU
    L.sbp_nn_gemm(M, N, K, Ad, lda, ta, Bd, ldb, tb, C, N, 0, bd, 1, 1.0, _stream())
    want = np.maximum(2 * ref, 0)
    assert np.abs(C.cpu().numpy() - want).max() < tol * np.abs(want).max()
    # BF16 output with ReLU
    Cb = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    L.sbp_nn_gemm(M, N, K, Ad, lda, ta, Bd, ldb, tb, Cb, N, 1, bd, 1, 0.0, _stream())
    want = np.maximum(ref, 0)
    assert np.abs(Cb.float().cpu().numpy() - want).max() < 1e-2 * np.abs(want).max()


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 512, 128), (200, 300, 100), (136, 200, 96), (40, 64, 1000),
                                   (1152, 2048, 640), (384, 640, 4096)])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_kernel_paths_vs_numpy(path, M, N, K, ta, tb):
    """Each GEMM kernel forced in turn: 1 the mma.sync kernels, 2 the tcgen05 kernel (TMA
    operand tiles in both orientations, FP32 accumulator in tensor memory, ragged M, N, K
    edges, split K for FP32 outputs that leave SMs idle).  Same tolerances as above; the
    tcgen05 kernel's status word stays clear."""
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    rng = np.random.default_rng(M + 3 * N + 7 * K + 11 * ta + 13 * tb)
    A = _bf(rng.normal(size=(K, M) if ta else (M, K)))
    B = _bf(rng.normal(size=(N, K) if tb else (K, N)))
    bias = torch.as_tensor(rng.normal(size=M), dtype=torch.float32)
    An = A.float().numpy().astype(np.float64)
    Bn = B.float().numpy().astype(np.float64)
    ref = (An.T if ta else An) @ (Bn.T if tb else Bn) + bias.numpy()[:, None]
    Ad, Bd, bd = A.cuda(), B.cuda(), bias.cuda()
    tol = 1e-5 * max(1.0, (K / 1024) ** 0.5)
    L.sbp_nn_set_gemm_path(path)
    try:
        C = torch.empty(M, N, device="cuda")
        L.sbp_nn_gemm(M, N, K, Ad, A.shape[1], ta, Bd, B.shape[1], tb, C, N, 0, bd, 0, 0.0, _stream())
        assert np.abs(C.cpu().numpy() - ref).max() < tol * np.abs(ref).max()
        L.sbp_nn_gemm(M, N, K, Ad, A.shape[1], ta, Bd, B.shape[1], tb, C, N, 0, bd, 1, 1.0, _stream())
        want = np.maximum(2 * ref, 0)
        assert np.abs(C.cpu().numpy() - want).max() < tol * np.abs(want).max()
        Cb = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
        L.sbp_nn_gemm(M, N, K, Ad, A.shape[1], ta, Bd, B.shape[1], tb, Cb, N, 1, bd, 1, 0.0, _stream())
        want = np.maximum(ref, 0)
        assert np.abs(Cb.float().cpu().numpy() - want).max() < 1e-2 * np.abs(want).max()
        assert L.sbp_nn_status() == 0
    finally:
        L.sbp_nn_set_gemm_path(0)


@pytest.mark.parametrize("n_mom", [0, 6])
def test_network_forward_and_gradients_vs_oracle(n_mom):
    from oracle import surrogate_net as sn
    from paper_2011_02600_gb300.surrogate import SurrogateNet, mse
    n_in, H, C, T0, n_up, n_out, B = 3, 48, 8, 4, 2, 6, 5
    net = SurrogateNet(n_in=n_in, hidden=H, C=C, T0=T0, n_up=n_up, n_out=n_out, n_mom=n_mom, seed=3)
    rng = np.random.default_rng(4)
    for n in net.names:   # non-zero biases so that every path is exercised
        net.b[n].copy_(torch.as_tensor(rng.normal(scale=0.1, size=net.b[n].numel()), dtype=torch.float32))
    x = _bf(rng.uniform(-1, 1, size=(n_in, B))).cuda()
    m = torch.as_tensor(rng.normal(size=(6, B)), dtype=torch.float32).cuda() if n_mom else None
    T = T0 * 2 ** n_up
    tgt = torch.as_tensor(rng.normal(size=(n_out, B * T)), dtype=torch.float32).cuda()
    y = net.forward(x, m, keep=True)
    loss, dy = mse(y, tgt)
    net.backward(dy)
    # oracle on the same BF16 weights (biases and m are FP32 in both)
    params = {n: (net.wb[n].float().cpu().numpy().astype(np.float64), net.b[n].cpu().numpy().astype(np.float64))
              for n in net.names}
    xo = x.float().cpu().numpy().astype(np.float64)
    mo = m.cpu().numpy().astype(np.float64) if n_mom else None
    to = tgt.cpu().numpy().reshape(n_out, B, T)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    for bf16, tol in ((True, 5e-3), (False, 1e-1)):
        yo, cache = sn.forward(params, xo, C, T0, n_up, m=mo, bf16=bf16)
        lo, dyo = sn.mse(yo, to)
        go = sn.backward(params, cache, dyo, C, T0, n_up)
        assert rel(y.cpu().numpy().reshape(n_out, B, T), yo) < tol / 2, bf16
        assert abs(loss - lo) < tol / 2 * lo, bf16
        for n in net.names:
            assert rel(net.gw[n].cpu().numpy(), go[n][0]) < tol, (n, bf16)
            assert rel(net.gb[n].cpu().numpy(), go[n][1]) < tol, (n, bf16)


def test_training_reduces_the_loss():
    from paper_2011_02600_gb300.surrogate import SurrogateNet, mse
    torch.manual_seed(0)
    net = SurrogateNet(n_in=7, hidden=64, C=16, T0=8, n_up=2, n_out=12, n_mom=0, seed=1)
    B = 32
    rng = np.random.default_rng(2)
    x = _bf(rng.uniform(-1, 1, size=(7, B))).cuda()
    T = 32
    t = torch.linspace(0, 1, T)
    tgt = torch.stack([torch.sin(6.28 * (k + 1) * t)[None, :].expand(B, T) for k in range(12)])
    tgt = (tgt * torch.as_tensor(rng.uniform(0.5, 1.5, size=(12, B, 1)), dtype=torch.float32)).reshape(12, -1)
    tgt = tgt.contiguous().cuda()
    losses = []
    for it in range(300):
        y = net.forward(x, keep=True)
        loss, dy = mse(y, tgt)
        net.backward(dy)
        net.adam(2e-3)
        losses.append(loss)
    assert losses[-1] < 0.05 * losses[0], (losses[0], losses[-1])


def test_surrogate_end_to_end_reduced():
    """Batched-solver data on a reduced configuration (33^3 nodes, order 4, 256 steps,
    0.5 Hz Ricker, 16 receivers, sources in a 4 x 4 x 2.25 km box of positions), training
    by the library's kernels, held-out error against the solver and speed-up.  The bar:
    the held-out median error is below half that of the best fit that ignores the source
    position (six trace sets fitted to all training samples by least squares)."""
    from paper_2011_02600_gb300 import surrogate as S
    from workloads.configs import config_by_name
    cfg = dataclasses.replace(config_by_name("surrogate97_o4"), nodes=(33, 33, 33), steps=256)
    lo = (0.4, 0.4, 0.65) + S.PARAM_LO[3:]
    hi = (0.6, 0.6, 0.8) + S.PARAM_HI[3:]
    n_train, n_test = 512, 128
    P = S.sample_params(0, n_train + n_test, lo, hi)
    Y, t_solve, info = S.generate_dataset(cfg, P, batch=64, f0=0.5, n_side=4)
    assert float(Y.abs().max()) > 0
    per = torch.as_tensor(S.M_REF / 10.0 ** P[:, 6], dtype=torch.float32, device=Y.device)[:, None, None]
    norm = float((Y[:n_train] * per[:n_train]).pow(2).mean().sqrt())
    net = S.SurrogateNet(n_in=3, hidden=512, C=128, T0=32, n_up=3, n_out=Y.shape[1], seed=0, lo=lo[:3], hi=hi[:3])
    losses = S.train(net, P[:n_train], (Y[:n_train] * per[:n_train] / norm).contiguous(), epochs=200, batch=32,
                     lr=1e-3)
    assert losses[-1] < 0.2 * losses[0]
    torch.cuda.synchronize()
    import time
    t0 = time.perf_counter()
    pred = S.predict(net, P[n_train:])
    torch.cuda.synchronize()
    t_net = (time.perf_counter() - t0) / n_test
    truth = Y[n_train:] / norm
    err = S.relative_l2(pred, truth)
    mt = S.moment_inputs(P[:n_train], unit=True).double()                  # [6][n]
    Yt = (Y[:n_train] * per[:n_train] / norm).double().reshape(n_train, -1)  # [n][F]
    G = torch.linalg.lstsq(mt.t(), Yt).solution                              # [6][F]
    mb = S.moment_inputs(P[n_train:]).double()
    base = S.relative_l2((mb.t() @ G).reshape(truth.shape).float(), truth)
    assert np.median(err) < 0.5 * np.median(base), (np.median(err), np.median(base))
    assert t_solve / t_net > 10, (t_solve, t_net)


def test_solver_fallback_outside_the_training_box():
    """Rows outside the box come from the batched solver (bitwise the dataset generator's
    traces); rows inside from the network times its scale."""
    from paper_2011_02600_gb300 import surrogate as S
    from workloads.configs import config_by_name
    cfg = dataclasses.replace(config_by_name("surrogate97_o4"), nodes=(25, 25, 25), steps=64)
    lo = (0.4, 0.4, 0.65) + S.PARAM_LO[3:]
    hi = (0.6, 0.6, 0.8) + S.PARAM_HI[3:]
    P = S.sample_params(1, 6)
    P[:3, :3] = S.sample_params(2, 3, lo, hi)[:, :3]
    P[3:, 0] = 0.25                                    # outside in q
    net = S.SurrogateNet(n_in=3, hidden=32, C=8, T0=8, n_up=3, n_out=3 * 9, seed=0, lo=lo[:3], hi=hi[:3])
    model = S.SeismogramModel(net, 2.5, cfg, f0=0.5, n_side=3, lo=lo, hi=hi, batch=4)
    y, by_solver = model.traces(P)
    assert list(by_solver) == [False] * 3 + [True] * 3
    want, _, _ = S.generate_dataset(cfg, P[3:], batch=3, f0=0.5, n_side=3)
    assert torch.equal(y[3:], want)
    assert torch.allclose(y[:3], S.predict(net, P[:3]) * 2.5)


@pytest.mark.parametrize("n_in,B,L", [(3, 37, 4), (3, 64, 6), (7, 5, 0)])
def test_fourier_features_kernel(n_in, B, L):
    """sbp_nn_fourier_features: x, then sin(2^k pi x), cos(2^k pi x) per input (BF16), as to_input
    forms the network's input."""
    from paper_2011_02600_gb300 import _lib as L_
    from paper_2011_02600_gb300.solver import _stream
    from paper_2011_02600_gb300.surrogate import to_input
    rng = np.random.default_rng(B + L)
    x = torch.as_tensor(rng.uniform(-1, 1, size=(n_in, B)), dtype=torch.float32).cuda()
    y = torch.empty(n_in * (1 + 2 * L), B, dtype=torch.bfloat16, device="cuda")
    L_.sbp_nn_fourier_features(x, y, n_in, B, L, _stream())
    xd = x.double().cpu().numpy()
    rows = [xd[i] for i in range(n_in)]
    for i in range(n_in):
        for k in range(L):
            rows += [np.sin(2.0 ** k * np.pi * xd[i]), np.cos(2.0 ** k * np.pi * xd[i])]
    want = np.stack(rows)
    assert np.abs(y.float().cpu().numpy() - want).max() <= 2.0 ** -7 * max(1.0, np.abs(want).max())
    # to_input: the normalised parameters' features
    P = rng.uniform(0.3, 0.7, size=(B, n_in))
    xb = to_input(P, [0.3] * n_in, [0.7] * n_in, L)
    assert xb.shape == (n_in * (1 + 2 * L), B)
    assert np.abs(xb[:n_in].float().cpu().numpy() - (5.0 * (P.T - 0.3) - 1.0)).max() < 1e-2
