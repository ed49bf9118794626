"""Pins of the oracle network: gradients against central finite differences (FP64),
the convolution against its direct sum, the moment combination against the
linearity it encodes, and the BF16 rounding against torch's conversion."""
import numpy as np
import pytest

from oracle import surrogate_net as sn


def _params(rng, n_in=3, H=6, C=2, T0=3, n_up=2, n_out=3):
    p = {"fc1": (rng.normal(size=(H, n_in)), rng.normal(size=H) * 0.1),
         "fc2": (rng.normal(size=(H, H)) / 2, rng.normal(size=H) * 0.1),
         "fc3": (rng.normal(size=(C * T0, H)) / 2, rng.normal(size=C * T0) * 0.1)}
    for i in range(n_up):
        p[f"conv{i}"] = (rng.normal(size=(C, C * 5)) / 3, rng.normal(size=C) * 0.1)
    p["out"] = (rng.normal(size=(n_out, C * 5)) / 3, rng.normal(size=n_out) * 0.1)
    return p


@pytest.mark.parametrize("moment", [False, True])
def test_backward_matches_finite_differences(moment):
    rng = np.random.default_rng(0)
    C, T0, n_up = 2, 3, 2
    p = _params(rng, C=C, T0=T0, n_up=n_up, n_out=18 if moment else 3)
    x = rng.normal(size=(3, 4))
    m = rng.normal(size=(6, 4)) if moment else None
    y, cache = sn.forward(p, x, C, T0, n_up, m=m)
    t = rng.normal(size=y.shape)
    loss, dy = sn.mse(y, t)
    g = sn.backward(p, cache, dy, C, T0, n_up)
    h = 1e-6
    for name in p:
        for which in (0, 1):
            arr = p[name][which]
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp, _ = sn.mse(sn.forward(p, x, C, T0, n_up, m=m)[0], t)
            arr[idx] = old - h
            lm, _ = sn.mse(sn.forward(p, x, C, T0, n_up, m=m)[0], t)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][which][idx]) < 1e-6 * max(1e-8, abs(fd)) + 1e-10, (name, which)


def test_conv_against_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 7))
    W = rng.normal(size=(4, 10))
    b = rng.normal(size=4)
    y = sn.conv1d(x, W, b)
    for o in range(4):
        for bb in range(3):
            for t in range(7):
                s = b[o]
                for c in range(2):
                    for k in range(5):
                        ts = t + k - 2
                        if 0 <= ts < 7:
                            s += W[o, c * 5 + k] * x[c, bb, ts]
                assert abs(s - y[o, bb, t]) < 1e-12


def test_moment_combination_is_the_weighted_sum_of_six_networks():
    """y(m) = sum_c m_c y_c where y_c is the network with only the c-th block of output rows."""
    rng = np.random.default_rng(2)
    C, T0, n_up, n_out = 2, 3, 1, 2
    p = _params(rng, C=C, T0=T0, n_up=n_up, n_out=6 * n_out)
    x = rng.normal(size=(3, 5))
    m = rng.normal(size=(6, 5))
    y, _ = sn.forward(p, x, C, T0, n_up, m=m)
    want = np.zeros_like(y)
    W, b = p["out"]
    for c in range(6):
        pc = dict(p)
        pc["out"] = (W[c * n_out:(c + 1) * n_out], b[c * n_out:(c + 1) * n_out])
        yc, _ = sn.forward(pc, x, C, T0, n_up)
        want += m[c][None, :, None] * yc
    assert np.abs(y - want).max() < 1e-12 * np.abs(want).max()


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        np.array([0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0e38])])
    want = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(sn.round_bf16(x), want)
