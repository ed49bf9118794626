"""The surrogate network in plain numpy FP64 (oracle for the BF16 tensor-core kernels).

Test infrastructure only; see ``oracle/__init__.py``.

The paper has no learned component; this is the textbook definition of the
network the library trains: fully connected layers y = W x + b with ReLU, a
reshape to channels x time, then [nearest x2 upsampling, 1D convolution
(width 5, zero padding 2), ReLU] blocks and a final linear convolution; the
loss is the mean squared error.  Backward is the chain rule written out layer
by layer.  Activations are [features][batch] and [channels][batch][time].

With moment components m ([6][batch]) the final convolution gives six trace sets
G_c ([6 * n_out] channels, c-major) and the output is y = sum_c m_c G_c: the
solver's receiver traces are linear in the six independent moment-tensor
components of the point source (Sec. 2 source term), so only the dependence on
the source position is learned.

``bf16=True`` rounds every value the library stores in BF16 (ReLU activations,
dL/dy and the ReLU-masked activation gradients) to BF16 at the same points,
round to nearest even from the FP32 value, so that the library's kernels can be
compared with it to FP32-accumulation accuracy.
"""
import numpy as np

KW, PAD = 5, 2


def round_bf16(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even) via FP32, as FP64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def _id(x):
    return x


def conv1d(x, W, b):
    """x [C][B][T], W [Co][C*KW] (index c*KW + k), b [Co] -> [Co][B][T]."""
    C, B, T = x.shape
    Co = W.shape[0]
    Wr = W.reshape(Co, C, KW)
    xp = np.zeros((C, B, T + 2 * PAD))
    xp[:, :, PAD:PAD + T] = x
    y = np.zeros((Co, B, T))
    for k in range(KW):
        y += np.einsum("oc,cbt->obt", Wr[:, :, k], xp[:, :, k:k + T])
    return y + b[:, None, None]


def conv1d_backward(x, W, dy):
    """Gradients (dx, dW, db) of conv1d."""
    C, B, T = x.shape
    Co = W.shape[0]
    Wr = W.reshape(Co, C, KW)
    xp = np.zeros((C, B, T + 2 * PAD))
    xp[:, :, PAD:PAD + T] = x
    dW = np.zeros_like(Wr)
    dxp = np.zeros_like(xp)
    for k in range(KW):
        dW[:, :, k] = np.einsum("obt,cbt->oc", dy, xp[:, :, k:k + T])
        dxp[:, :, k:k + T] += np.einsum("oc,obt->cbt", Wr[:, :, k], dy)
    return dxp[:, :, PAD:PAD + T], dW.reshape(Co, C * KW), dy.sum(axis=(1, 2))


def forward(params, x, C, T0, n_up, m=None, bf16=False):
    """params: dict name -> (W, b); x [n_in][B]; m [6][B] or None.
    Returns (y [n_out][B][T], cache)."""
    rb = round_bf16 if bf16 else _id
    relu = lambda z: rb(np.maximum(z, 0.0))
    cache = {"x": x, "m": m, "bf16": bf16}
    h = x
    for name in ("fc1", "fc2", "fc3"):
        W, b = params[name]
        z = W @ h + b[:, None]
        cache[name] = (h, z)
        h = relu(z)
    B = x.shape[1]
    a = h.reshape(C, T0, B).transpose(0, 2, 1)          # [c][b][t]
    cache["a0"] = a
    for i in range(n_up):
        u = np.repeat(a, 2, axis=2)
        W, b = params[f"conv{i}"]
        z = conv1d(u, W, b)
        cache[f"conv{i}"] = (u, z)
        a = relu(z)
    W, b = params["out"]
    y = conv1d(a, W, b)
    cache["out"] = (a, y)
    if m is not None:
        G = rb(y.reshape(6, -1, *y.shape[1:]))   # the six trace sets, stored in BF16 like the activations
        y = np.einsum("cb,cobt->obt", m, G)
    return y, cache


def backward(params, cache, dy, C, T0, n_up):
    """Gradients dict name -> (dW, db) given dL/dy [n_out][B][T]."""
    rb = round_bf16 if cache["bf16"] else _id
    dy = rb(dy)
    if cache["m"] is not None:
        dy = rb(np.einsum("cb,obt->cobt", cache["m"], dy).reshape(-1, *dy.shape[1:]))
    g = {}
    a, _ = cache["out"]
    da, dW, db = conv1d_backward(a, params["out"][0], dy)
    g["out"] = (dW, db)
    for i in reversed(range(n_up)):
        u, z = cache[f"conv{i}"]
        dz = rb(da * (z > 0))
        du, dW, db = conv1d_backward(u, params[f"conv{i}"][0], dz)
        g[f"conv{i}"] = (dW, db)
        C_, B, T2 = du.shape
        da = du.reshape(C_, B, T2 // 2, 2).sum(axis=3)
    B = da.shape[1]
    dh = da.transpose(0, 2, 1).reshape(C * T0, B)
    for name in ("fc3", "fc2", "fc1"):
        hin, z = cache[name]
        dz = rb(dh * (z > 0))
        W = params[name][0]
        g[name] = (dz @ hin.T, dz.sum(axis=1))
        dh = W.T @ dz
    return g


def mse(y, t):
    """(loss, dL/dy) of the mean squared error."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size
