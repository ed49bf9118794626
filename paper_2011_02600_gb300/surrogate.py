"""Learned surrogate of the solver: source parameters -> receiver traces.

Network (BF16 weights and activations, FP32 accumulation on tensor cores):
    x (normalised source position q, r, s), with n_freq > 0 followed by its Fourier features
    sin(2^k pi x), cos(2^k pi x), k < n_freq (sbp_nn_fourier_features)
    -> 3 fully connected layers with ReLU (3 -> H -> H -> C*T0), reshaped to C channels x T0 samples
    -> n_up times [nearest x2 upsampling in time, 1D convolution (width 5) C -> C, ReLU]
    -> 1D convolution (width 5) C -> 6 * n_out, linear: six trace sets G_c
    -> y = sum_c m_c G_c with m the six Voigt moment-tensor components of the source
giving 3 velocity components at every receiver (n_out = 3 * n_receivers) for
T0 * 2**n_up time samples.  The solver is linear in the source term, so the
traces are exactly linear in the moment tensor: only the dependence on the
source position is learned, and strike, dip, rake and M0 enter through m.

Every layer runs in the library's kernels (sbp_nn_*): GEMMs on BF16 tensor cores,
im2col/col2im for the convolutions, ReLU masks, bias gradients, the MSE loss and
Adam on FP32 master weights.  Torch only allocates the buffers.

Activations of a batch of B samples are stored feature-major: [features][B] for
the fully connected part and [channels][B * T] for the convolutions.

The training data come from the batched solver (one source per batch member, see
``generate_dataset``); the solver also judges the network's error and is the
fallback for parameters outside the training box.
"""
import math
import time

import numpy as np
import torch

from . import _lib as L
from .solver import _stream

KW = 5
PAD = 2


class SurrogateNet:
    def __init__(self, n_in=3, hidden=512, C=128, T0=32, n_up=5, n_out=192, n_mom=6, seed=0, device="cuda",
                 lo=None, hi=None, n_freq=0):
        """n_mom = 6: moment-linear output (forward needs m); n_mom = 0: the last layer is the output.
        lo, hi: the box of source positions (q, r, s) the network is trained on; inputs are
        mapped from it to [-1, 1]."""
        if n_mom not in (0, 6):
            raise ValueError("n_mom must be 0 or 6")
        self.lo = tuple(lo if lo is not None else PARAM_LO[:n_in])
        self.hi = tuple(hi if hi is not None else PARAM_HI[:n_in])
        self.n_in, self.hidden, self.C, self.T0, self.n_up, self.n_out = n_in, hidden, C, T0, n_up, n_out
        self.n_mom = n_mom
        self.n_freq = n_freq
        self.n_feat = n_in * (1 + 2 * n_freq)   # the first layer's inputs
        self.n_last = n_out * max(1, n_mom)
        self.T = T0 * 2 ** n_up
        self.device = torch.device(device)
        g = torch.Generator(device="cpu").manual_seed(seed)
        shapes = [("fc1", hidden, self.n_feat), ("fc2", hidden, hidden), ("fc3", C * T0, hidden)]
        shapes += [(f"conv{i}", C, C * KW) for i in range(n_up)]
        shapes += [("out", self.n_last, C * KW)]
        self.names = [s[0] for s in shapes]
        self.w, self.b, self.wb = {}, {}, {}
        self.gw, self.gb = {}, {}
        self.mw, self.vw, self.mb, self.vb = {}, {}, {}, {}
        for name, o, i in shapes:
            std = math.sqrt(2.0 / i) if name != "out" else math.sqrt(1.0 / i)
            w = (torch.randn(o, i, generator=g, dtype=torch.float64) * std).float().to(self.device)
            self.w[name] = w
            self.b[name] = torch.zeros(o, device=self.device)
            self.wb[name] = w.to(torch.bfloat16)
            for d in (self.gw, self.mw, self.vw):
                d[name] = torch.zeros_like(w)
            for d in (self.gb, self.mb, self.vb):
                d[name] = torch.zeros(o, device=self.device)
        self.step_count = 0
        self.cache = {}

    # ---- helpers -------------------------------------------------------------
    @staticmethod
    def _gemm(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, bf16_out, bias=None, relu=0, beta=0.0):
        L.sbp_nn_gemm(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, 1 if bf16_out else 0, bias, relu, beta, _stream())

    def n_params(self):
        return sum(self.w[n].numel() + self.b[n].numel() for n in self.names)

    # ---- forward -------------------------------------------------------------
    def forward(self, x, m=None, keep=False):
        """x: BF16 [n_feat][B] (normalised parameters and their Fourier features: to_input);
        m: FP32 [6][B] moment components
        (n_mom = 6).  Returns FP32 [n_out][B * T]."""
        if (m is None) != (self.n_mom == 0):
            raise ValueError("m must be given exactly when n_mom = 6")
        B = x.shape[1]
        dev = self.device
        bf = dict(dtype=torch.bfloat16, device=dev)
        H, C, T0 = self.hidden, self.C, self.T0
        h1 = torch.empty(H, B, **bf)
        self._gemm(H, B, self.n_feat, self.wb["fc1"], self.n_feat, 0, x, B, 0, h1, B, True, self.b["fc1"], 1)
        h2 = torch.empty(H, B, **bf)
        self._gemm(H, B, H, self.wb["fc2"], H, 0, h1, B, 0, h2, B, True, self.b["fc2"], 1)
        h3 = torch.empty(C * T0, B, **bf)
        self._gemm(C * T0, B, H, self.wb["fc3"], H, 0, h2, B, 0, h3, B, True, self.b["fc3"], 1)
        a = torch.empty(C, B * T0, **bf)
        L.sbp_nn_mlp_to_conv(h3, a, C, T0, B, 0, _stream())
        acts = [a]
        cols = []
        T = T0
        for i in range(self.n_up):
            u = torch.empty(C, B * 2 * T, **bf)
            L.sbp_nn_upsample2(a, u, C * B, T, 0, _stream())
            T *= 2
            col = torch.empty(C * KW, B * T, **bf)
            L.sbp_nn_im2col(u, col, C, B, T, KW, PAD, _stream())
            a = torch.empty(C, B * T, **bf)
            self._gemm(C, B * T, C * KW, self.wb[f"conv{i}"], C * KW, 0, col, B * T, 0, a, B * T, True,
                       self.b[f"conv{i}"], 1)
            acts.append(a)
            cols.append(col)
        col = torch.empty(C * KW, B * T, **bf)
        L.sbp_nn_im2col(a, col, C, B, T, KW, PAD, _stream())
        # the six trace sets in BF16 like the other activations (the traces y combined from them
        # are FP32); the output itself (n_mom = 0) in FP32
        g = torch.empty(self.n_last, B * T, dtype=torch.bfloat16 if self.n_mom else torch.float32, device=dev)
        self._gemm(self.n_last, B * T, C * KW, self.wb["out"], C * KW, 0, col, B * T, 0, g, B * T,
                   bool(self.n_mom), self.b["out"], 0)
        y = g
        if self.n_mom:
            y = torch.empty(self.n_out, B * T, dtype=torch.float32, device=dev)
            L.sbp_nn_moment_combine(g, m, y, None, None, self.n_out, B, T, 0, _stream())
        if keep:
            self.cache = dict(B=B, x=x, m=m, h1=h1, h2=h2, h3=h3, acts=acts, cols=cols, col_out=col)
        return y

    # ---- backward ------------------------------------------------------------
    def backward(self, dy):
        """dy: BF16 [n_out][B * T] (dLoss/dy).  Fills self.gw / self.gb (FP32)."""
        c = self.cache
        B = c["B"]
        dev = self.device
        bf = dict(dtype=torch.bfloat16, device=dev)
        f32 = dict(dtype=torch.float32, device=dev)
        C, T0, H = self.C, self.T0, self.hidden
        T = self.T
        N = B * T
        st = _stream()
        if self.n_mom:
            dg = torch.empty(self.n_last, N, **bf)
            L.sbp_nn_moment_combine(None, c["m"], None, dy, dg, self.n_out, B, T, 1, st)
            dy = dg
        # output layer
        self._gemm(self.n_last, C * KW, N, dy, N, 0, c["col_out"], N, 1, self.gw["out"], C * KW, False)
        L.sbp_nn_bias_grad(dy, self.gb["out"], self.n_last, N, st)
        dcol = torch.empty(C * KW, N, **f32)
        self._gemm(C * KW, N, self.n_last, self.wb["out"], C * KW, 1, dy, N, 0, dcol, N, False)
        da = torch.empty(C, N, **f32)
        L.sbp_nn_col2im(dcol, da, C, B, T, KW, PAD, st)
        for i in reversed(range(self.n_up)):
            a = c["acts"][i + 1]
            dz = torch.empty(C, B * T, **bf)
            L.sbp_nn_relu_backward(da, a, dz, C * B * T, st)
            col = c["cols"][i]
            self._gemm(C, C * KW, B * T, dz, B * T, 0, col, B * T, 1, self.gw[f"conv{i}"], C * KW, False)
            L.sbp_nn_bias_grad(dz, self.gb[f"conv{i}"], C, B * T, st)
            dcol = torch.empty(C * KW, B * T, **f32)
            self._gemm(C * KW, B * T, C, self.wb[f"conv{i}"], C * KW, 1, dz, B * T, 0, dcol, B * T, False)
            du = torch.empty(C, B * T, **f32)
            L.sbp_nn_col2im(dcol, du, C, B, T, KW, PAD, st)
            T //= 2
            da = torch.empty(C, B * T, **f32)
            L.sbp_nn_upsample2(du, da, C * B, T, 1, st)
        # fully connected part (a0 is h3 reshaped)
        dz = torch.empty(C, B * T0, **bf)
        L.sbp_nn_relu_backward(da, c["acts"][0], dz, C * B * T0, st)
        dh3 = torch.empty(C * T0, B, **bf)
        L.sbp_nn_mlp_to_conv(dh3, dz, C, T0, B, 1, st)
        self._fc_backward("fc3", dh3, c["h2"], C * T0, H, B)
        dh2 = torch.empty(H, B, **f32)
        self._gemm(H, B, C * T0, self.wb["fc3"], H, 1, dh3, B, 0, dh2, B, False)
        dz2 = torch.empty(H, B, **bf)
        L.sbp_nn_relu_backward(dh2, c["h2"], dz2, H * B, st)
        self._fc_backward("fc2", dz2, c["h1"], H, H, B)
        dh1 = torch.empty(H, B, **f32)
        self._gemm(H, B, H, self.wb["fc2"], H, 1, dz2, B, 0, dh1, B, False)
        dz1 = torch.empty(H, B, **bf)
        L.sbp_nn_relu_backward(dh1, c["h1"], dz1, H * B, st)
        self._fc_backward("fc1", dz1, c["x"], H, self.n_feat, B)

    def _fc_backward(self, name, dz, xin, o, i, B):
        self._gemm(o, i, B, dz, B, 0, xin, B, 1, self.gw[name], i, False)
        L.sbp_nn_bias_grad(dz, self.gb[name], o, B, _stream())

    # ---- optimiser -----------------------------------------------------------
    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        st = _stream()
        for n in self.names:
            L.sbp_nn_adam(self.w[n], self.gw[n], self.mw[n], self.vw[n], self.wb[n], self.w[n].numel(), lr, b1, b2,
                          eps, self.step_count, st)
            L.sbp_nn_adam(self.b[n], self.gb[n], self.mb[n], self.vb[n], None, self.b[n].numel(), lr, b1, b2, eps,
                          self.step_count, st)


def mse(y, target, want_grad=True, nblocks=256):
    """(loss, dL/dy BF16) of the mean squared error, by the library's loss kernel."""
    n = y.numel()
    partial = torch.zeros(nblocks, dtype=torch.float64, device=y.device)
    dy = torch.empty_like(y, dtype=torch.bfloat16) if want_grad else None
    L.sbp_nn_mse(y, target, dy, n, partial, nblocks, _stream())
    return float(partial.sum()) / n, dy


def to_input(params, lo, hi, n_freq=0):
    """Normalise [B][n_in] position parameters to [-1, 1] and form the network's BF16
    [n_in (1 + 2 n_freq)][B] input (the parameters and their Fourier features, in the library)."""
    p = torch.as_tensor(params, dtype=torch.float32)
    x = (2.0 * (p - torch.as_tensor(lo, dtype=torch.float32)) /
         torch.as_tensor(np.asarray(hi) - np.asarray(lo), dtype=torch.float32) - 1.0).t().contiguous()
    x = x.cuda()
    n_in, B = x.shape
    xb = torch.empty(n_in * (1 + 2 * n_freq), B, dtype=torch.bfloat16, device=x.device)
    L.sbp_nn_fourier_features(x, xb, n_in, B, n_freq, _stream())
    return xb


# ---------------------------------------------------------------------------------------------
# Training data from the batched solver

PARAM_NAMES = ("q", "r", "s", "strike", "dip", "rake", "log10_M0")
PARAM_LO = (0.3, 0.3, 0.6, 0.0, 0.3, -math.pi, 14.0)
PARAM_HI = (0.7, 0.7, 0.85, 2 * math.pi, math.pi / 2, math.pi, 16.0)
M_REF = 1e15     # moment of the unit the network's traces are expressed in (N m)


def moment_inputs(params, unit=False):
    """FP32 [6][B] Voigt moment components for parameter rows (device): in units of M_REF,
    or of each row's own M0 (unit=True, the moment tensor of a unit-moment source)."""
    from .source_util import moment_tensor_voigt
    m = np.array([moment_tensor_voigt(p[3], p[4], p[5], 1.0 if unit else 10.0 ** (p[6] - math.log10(M_REF)))
                  for p in params])
    return torch.as_tensor(m.T.copy(), dtype=torch.float32).cuda()


def sample_params(seed, n, lo=PARAM_LO, hi=PARAM_HI):
    """n parameter rows drawn uniformly from the box [lo, hi] (seeded)."""
    rng = np.random.default_rng([seed, 6006])
    return np.stack([rng.uniform(a, b, n) for a, b in zip(lo, hi)], axis=1)


def generate_dataset(cfg, params, batch=64, f0=None, n_side=8, precision=32, every=1):
    """Traces [n][3 * n_rec][T] (FP32, device) of the batched solver for each parameter row
    (reference position q, r, s; strike, dip, rake; log10 M0), sampled every ``every``
    steps (T = cfg.steps / every), plus the solver time per sample (seconds) and the
    solver's (dt, hmin, cpmax)."""
    if cfg.steps % every:
        raise ValueError("the step count must be a multiple of the sampling interval")
    from workloads.acquisition import surface_receivers
    from .source_util import moment_tensor_voigt
    from .workload_setup import build_solver
    n = len(params)
    T = cfg.steps
    f0 = f0 or cfg.extra.get("f0", 2.0)
    rec = surface_receivers(cfg.nodes, n_side)
    out = torch.empty(n, 3 * len(rec), T // every, dtype=torch.float32, device="cuda")
    s, info = build_solver(cfg, precision=precision, keep_metrics=True, batch=batch)
    tr = s.set_receivers(rec, T)
    t_solve = 0.0
    for b0 in range(0, n, batch):
        chunk = params[b0:b0 + batch]
        srcs = []
        for p in chunk:
            Mv = moment_tensor_voigt(p[3], p[4], p[5], 10.0 ** p[6])
            srcs.append(dict(ref=(float(p[0]), float(p[1]), float(p[2])), moment=list(Mv)))
        while len(srcs) < batch:  # pad the last batch with silent sources
            srcs.append(dict(ref=srcs[0]["ref"], moment=[0.0] * 6))
        s.set_sources(srcs, f0=f0)
        for qb in s.qbuf:
            qb.zero_()
        s.dq.zero_()
        s.set_time(0.0, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(T, info["dt"])
        torch.cuda.synchronize()
        t_solve += time.perf_counter() - t0
        m = len(chunk)
        out[b0:b0 + m] = tr[:m].reshape(m, -1, T)[:, :, every - 1::every].float()
    return out, t_solve / n, info


def train(net, X, Y, epochs, batch=32, lr=1e-3, seed=0, log_every=0):
    """X: [n][7] params (numpy); Y: [n][n_out][T] FP32 traces of each row divided by its
    M0 / M_REF and by one global scale (device).  The moment input is the unit-moment
    tensor, so every sample weighs alike in the loss whatever its M0.  Returns the mean
    loss per epoch."""
    n = len(X)
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        perm = rng.permutation(n)
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        tot = 0.0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            x = to_input(X[idx, :net.n_in], net.lo, net.hi, net.n_freq)
            m = moment_inputs(X[idx], unit=True) if net.n_mom else None
            tgt = Y[torch.as_tensor(idx, device=Y.device)].permute(1, 0, 2).reshape(net.n_out, -1).contiguous()
            y = net.forward(x, m, keep=True)
            loss, dy = mse(y, tgt)
            net.backward(dy)
            net.adam(lr_ep)
            tot += loss
        losses.append(tot / max(1, n // batch))
        if log_every and ep % log_every == 0:
            print(f"epoch {ep} loss {losses[-1]:.4e}", flush=True)
    return losses


def predict(net, X, batch=64):
    """Network traces [n][n_out][T] (FP32) for parameter rows X, in the units of the
    solver's traces divided by the training's global scale."""
    outs = []
    for b0 in range(0, len(X), batch):
        x = to_input(X[b0:b0 + batch, :net.n_in], net.lo, net.hi, net.n_freq)
        y = net.forward(x, moment_inputs(X[b0:b0 + batch]) if net.n_mom else None)
        B = x.shape[1]
        outs.append(y.view(net.n_out, B, net.T).permute(1, 0, 2))
    return torch.cat(outs)


def relative_l2(pred, true):
    """Per-sample ||pred - true|| / ||true||."""
    d = (pred - true).reshape(len(true), -1).double()
    t = true.reshape(len(true), -1).double()
    return (d.norm(dim=1) / t.norm(dim=1)).cpu().numpy()


# ---------------------------------------------------------------------------------------------
# Network with the solver as fallback, and the full workload

def in_box(params, lo=PARAM_LO, hi=PARAM_HI):
    """Mask of parameter rows inside the training box (all 7 parameters)."""
    p = np.asarray(params)
    return np.all((p >= np.asarray(lo)) & (p <= np.asarray(hi)), axis=1)


class SeismogramModel:
    """Traces for source parameters: the trained network inside its training box, the
    batched solver outside it.  ``norm`` converts network units to the solver's traces."""

    def __init__(self, net, norm, cfg, f0, n_side, every=1, lo=PARAM_LO, hi=PARAM_HI, batch=64):
        self.net, self.norm, self.cfg, self.f0, self.n_side, self.every = net, float(norm), cfg, f0, n_side, every
        self.lo, self.hi, self.batch = tuple(lo), tuple(hi), batch

    def traces(self, params):
        """[n][3 * n_rec][T] FP32 device traces and the mask of rows the solver computed."""
        params = np.asarray(params, dtype=np.float64)
        inside = in_box(params, self.lo, self.hi)
        out = torch.empty(len(params), self.net.n_out, self.net.T, dtype=torch.float32, device="cuda")
        if inside.any():
            out[torch.as_tensor(np.nonzero(inside)[0], device="cuda")] = predict(self.net, params[inside]) * self.norm
        if (~inside).any():
            y, _, _ = generate_dataset(self.cfg, params[~inside], batch=min(self.batch, int((~inside).sum())),
                                       f0=self.f0, n_side=self.n_side, every=self.every)
            out[torch.as_tensor(np.nonzero(~inside)[0], device="cuda")] = y
        return out, ~inside


def make_dataset(cfg, n_train=None, n_test=None, seed=0, gen_batch=64, log=print):
    """The workload's training and held-out sources (seeded) and their traces from the batched
    solver: (P [n][7], Y [n][n_out][T] FP32 device, info dict)."""
    n_train = n_train or cfg.extra["n_train"]
    n_test = n_test or cfg.extra["n_test"]
    T = cfg.extra.get("n_samples", cfg.steps)
    every = cfg.steps // T
    f0, n_side = cfg.extra["f0"], cfg.extra.get("n_side", 8)
    P = sample_params(seed, n_train + n_test)
    t0 = time.perf_counter()
    Y, t_solve, _ = generate_dataset(cfg, P, batch=gen_batch, f0=f0, n_side=n_side, every=every)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    if log:
        log(f"dataset {tuple(Y.shape)} in {t_gen:.1f} s, solver {t_solve * 1e3:.2f} ms per source")
    return P, Y, dict(n_train=n_train, n_test=n_test, samples=T, f0=f0, dataset_s=t_gen, solver_s=t_solve)


def train_and_judge(cfg, P, Y, info, epochs=200, batch=32, lr=1e-3, hidden=512, C=128, T0=32, n_freq=0, seed=0,
                    log=print):
    """Train the network on the first n_train sources with the library's kernels and judge it
    against the solver's traces of the held-out ones.  Returns sizes, timings, errors and the
    speed-up."""
    n_train, n_test, T = info["n_train"], info["n_test"], info["samples"]
    n_up = int(round(math.log2(T / T0)))
    if T0 * 2 ** n_up != T:
        raise ValueError("samples per trace must be T0 times a power of two")
    per = torch.as_tensor(M_REF / 10.0 ** P[:, 6], dtype=torch.float32, device=Y.device)[:, None, None]
    Yt = Y[:n_train] * per[:n_train]
    norm = float(Yt.pow(2).mean().sqrt())
    Yt /= norm
    net = SurrogateNet(n_in=3, hidden=hidden, C=C, T0=T0, n_up=n_up, n_out=Y.shape[1], seed=seed, n_freq=n_freq)
    t0 = time.perf_counter()
    losses = train(net, P[:n_train], Yt, epochs=epochs, batch=batch, lr=lr, seed=seed,
                   log_every=max(1, epochs // 10) if log else 0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del Yt
    predict(net, P[n_train:n_train + 1])      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pred = predict(net, P[n_train:], batch=64)
    torch.cuda.synchronize()
    t_net = (time.perf_counter() - t0) / n_test
    truth = Y[n_train:] / norm
    err = relative_l2(pred, truth)
    mt = moment_inputs(P[:n_train], unit=True).double()
    G = torch.linalg.lstsq(mt.t(), (Y[:n_train] * per[:n_train] / norm).double().reshape(n_train, -1)).solution
    base = relative_l2((moment_inputs(P[n_train:]).double().t() @ G).reshape(truth.shape).float(), truth)
    t_solve = info["solver_s"]
    return dict(nodes=list(cfg.nodes), order=cfg.order, steps=cfg.steps, samples=T, receivers=Y.shape[1] // 3,
                f0=info["f0"], n_train=n_train, n_test=n_test, epochs=epochs, hidden=hidden, n_freq=n_freq,
                params=net.n_params(), dataset_s=info["dataset_s"], train_s=t_train,
                solver_ms_per_source=t_solve * 1e3, net_ms_per_source=t_net * 1e3, speedup=t_solve / t_net,
                err_median=float(np.median(err)), err_p90=float(np.quantile(err, 0.9)),
                position_blind_err_median=float(np.median(base)), loss_first=losses[0], loss_last=losses[-1])


def run_workload(cfg, n_train=None, n_test=None, epochs=200, batch=32, lr=1e-3, hidden=512, C=128, T0=32,
                 seed=0, gen_batch=64, n_freq=0, log=print):
    """Generate the workload's training and held-out sets with the batched solver, train the
    network with the library's kernels, and judge it against the solver on the held-out
    sources.  Returns a dict of sizes, timings, errors and the speed-up."""
    P, Y, info = make_dataset(cfg, n_train, n_test, seed=seed, gen_batch=gen_batch, log=log)
    return train_and_judge(cfg, P, Y, info, epochs=epochs, batch=batch, lr=lr, hidden=hidden, C=C, T0=T0,
                           n_freq=n_freq, seed=seed, log=log)


def main(argv=None):
    import argparse
    import json
    from workloads.configs import config_by_name
    ap = argparse.ArgumentParser(description="Train and judge the surrogate on the 97^3 surrogate workload")
    ap.add_argument("--n-train", type=int, default=None)
    ap.add_argument("--n-test", type=int, default=None)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--n-freq", type=int, default=0, help="Fourier features of the position input (0: none)")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    res = run_workload(config_by_name("surrogate97_o4"), a.n_train, a.n_test, epochs=a.epochs, lr=a.lr,
                       hidden=a.hidden, n_freq=a.n_freq)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
