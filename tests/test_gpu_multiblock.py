"""Two blocks coupled at a shared face (multiblock.py; Section 7.1's two-block LOH1 setup) on
the GPU, through the C ABI (SBP_BC_INTERFACE, sbp_interface_trace, sbp_set_interface).

* The right-hand sides of both blocks against the oracle's two-block scheme
  (oracle/multiblock.py): 1e-12 in FP64, 5e-5 in FP32 (the tolerances of test_gpu_parity.py),
  curved blocks and a curved interface, random media on each side, the shared face on each of
  the three axes, tiled and general kernels.
* Energy: with free surfaces on every outer face, <Q, P~^-1 dQ/dt>_H of the GPU's right-hand
  sides equals the oracle's interface dissipation (the coupled scheme's energy identity), and
  the energy of a run never grows.
* A plane SH wave crossing a flat interface between two homogeneous media: the transmitted and
  reflected pulses have the textbook amplitudes 2 Z1 / (Z1 + Z2) and (Z1 - Z2) / (Z1 + Z2) of the
  incident one (Z = rho c_s), to 1 %."""
import math

import numpy as np
import pytest
import torch

from oracle import multiblock as MB
from oracle.elastic import Scheme
from oracle.metrics import metrics
from workloads.fields import random_state
from workloads.twoblock import block_coordinates, two_block_maps

pytestmark = pytest.mark.gpu

FREE = [("free",)] * 6


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _maps(xi, d=0.05, warp=0.2):
    fm, fp = two_block_maps(700.0, 1100.0, 1200.0, 900.0, d=d * 1000.0, warp=warp)
    if xi == 0:
        return fm, fp

    def wrap(f):   # the shared face on axis xi: swap q with axis xi and x with the same coordinate
        def g(q, r, s):
            a = [q, r, s]
            a[0], a[xi] = a[xi], a[0]
            x = list(f(*a))
            x[0], x[xi] = x[xi], x[0]
            return tuple(x)
        return g
    return wrap(fm), wrap(fp)


def _nodes(xi, through_m, through_p, other=(17, 16)):
    nm, npl = [other[0], other[0], other[1]], [other[0], other[0], other[1]]
    tang = [a for a in range(3) if a != xi]
    nm[tang[0]], nm[tang[1]] = other
    npl[tang[0]], npl[tang[1]] = other
    nm[xi], npl[xi] = through_m, through_p
    return tuple(nm), tuple(npl)


def _medium(shape, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(1500.0, 2500.0, shape)
    mu = rng.uniform(2.0e9, 6.0e9, shape)
    lam = rng.uniform(1.0e9, 8.0e9, shape)
    return rho, lam, mu


def _case(order, xi, operator="upwind"):
    nm, npl = _nodes(xi, 19, 23)
    fm, fp = _maps(xi)
    Xm, Xp = block_coordinates(fm, nm), block_coordinates(fp, npl)
    Jm, am = metrics(*Xm, order)
    Jp, ap = metrics(*Xp, order)
    assert Jm.min() > 0 and Jp.min() > 0
    return nm, npl, Xm, Xp, Jm, am, Jp, ap, Scheme(order, nm, operator), Scheme(order, npl, operator)


def _relerr(got, want):
    got = np.asarray(got, dtype=float)
    axes = tuple(range(1, want.ndim))
    return (np.abs(got - want).max(axis=axes) / np.maximum(np.abs(want).max(axis=axes), 1e-300)).max()


def _solver(nm, npl, order, prec, bc_m, bc_p, xi, Xm, Xp, mat_m, mat_p, operator="upwind"):
    from paper_2011_02600_gb300.multiblock import TwoBlockSolver
    tb = TwoBlockSolver(nm, npl, order, prec, bc_m, bc_p, xi=xi, operator=operator)
    tb.setup(torch.from_numpy(np.stack(Xm)), torch.from_numpy(np.stack(mat_m)),
             torch.from_numpy(np.stack(Xp)), torch.from_numpy(np.stack(mat_p)))
    return tb


def _smooth(X, seed):
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 2.0, size=(9, 3)) * 2 * math.pi / 2000.0
    ph = rng.uniform(0, 2 * math.pi, size=9)
    amp = np.array([1.0] * 3 + [1.0e6] * 6)
    return np.stack([amp[c] * np.sin(k[c, 0] * X[0] + k[c, 1] * X[1] + k[c, 2] * X[2] + ph[c]) for c in range(9)])


@pytest.mark.parametrize("order,operator,xi", [(4, "upwind", 0), (6, "upwind", 0), (4, "upwind", 1), (6, "upwind", 2),
                                               (2, "upwind", 0), (3, "upwind", 1), (4, "traditional", 2)])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("path", [0, 1])
def test_two_block_rhs_matches_oracle(order, operator, xi, prec, path):
    nm, npl, Xm, Xp, Jm, am, Jp, ap, sm, sp = _case(order, xi, operator)
    mat_m, mat_p = _medium(Jm.shape, 1), _medium(Jp.shape, 2)
    bc_m = [("char", 0.0), ("free",), ("char", 0.3), ("free",), ("char", -0.2), ("free",)]
    bc_p = [("free",), ("char", 0.0), ("free",), ("char", 0.5), ("free",), ("char", 0.0)]
    bc_m[2 * xi + 1] = ("interface",)
    bc_p[2 * xi] = ("interface",)
    if prec == 64:
        Qm, Qp = random_state(nm, 3, 1.0, 1.0e6), random_state(npl, 4, 1.0, 1.0e6)
    else:
        Qm, Qp = _smooth(Xm, 5), _smooth(Xp, 5)
    want_m, want_p = MB.two_block_rhs(Qm, Qp, sm, sp, Jm, Jp, am, ap, mat_m, mat_p, bc_m, bc_p, xi)
    tb = _solver(nm, npl, order, prec, bc_m, bc_p, xi, Xm, Xp, mat_m, mat_p, operator)
    tb.m.set_kernel_path(path)
    tb.p.set_kernel_path(path)
    got_m, got_p = (g.cpu().numpy() for g in tb.rhs(Qm, Qp))
    tol = 1e-12 if prec == 64 else 5e-5
    assert _relerr(got_m, want_m) < tol
    assert _relerr(got_p, want_p) < tol


def test_energy_identity_and_decay_on_the_gpu():
    order, xi = 6, 0
    nm, npl, Xm, Xp, Jm, am, Jp, ap, sm, sp = _case(order, xi)
    mat_m, mat_p = _medium(Jm.shape, 1), _medium(Jp.shape, 2)
    bc_m, bc_p = list(FREE), list(FREE)
    bc_m[1], bc_p[0] = ("interface",), ("interface",)
    Qm, Qp = random_state(nm, 7, 1.0, 1.0e6), random_state(npl, 8, 1.0, 1.0e6)
    tb = _solver(nm, npl, order, 64, bc_m, bc_p, xi, Xm, Xp, mat_m, mat_p)
    dm, dp = (g.cpu().numpy() for g in tb.rhs(Qm, Qp))

    def rate(Q, d, J, mat, sch):   # <Q, P~^-1 dQ/dt>_H from the GPU's dQ/dt
        rho, lam, mu = mat
        W = sch.weights3()
        pv = sum(Q[c] * rho * J * d[c] for c in range(3))
        ds = d[3:9]
        tr = ds[0] + ds[1] + ds[2]
        Sd = [(ds[c] - lam / (3 * lam + 2 * mu) * tr) / (2 * mu) for c in range(3)] + [ds[c] / mu for c in range(3, 6)]
        ps = sum(Q[3 + c] * J * Sd[c] for c in range(6))
        return float(np.sum(W * (pv + ps)))
    got = rate(Qm, dm, Jm, mat_m, sm) + rate(Qp, dp, Jp, mat_p, sp)
    _, want, _ = MB.interface_energy_rate(Qm, Qp, sm, sp, am, ap, mat_m, mat_p, bc_m, bc_p, xi)
    assert want < 0 and abs(got - want) < 1e-10 * abs(want)
    tb.m.set_state(torch.from_numpy(_smooth(Xm, 9)))
    tb.p.set_state(torch.from_numpy(_smooth(Xp, 10)))
    E = [tb.energy()]
    cmax = math.sqrt(max((mat_m[1] + 2 * mat_m[2]).max() / mat_m[0].min(), (mat_p[1] + 2 * mat_p[2]).max() / mat_p[0].min()))
    dt = 0.25 * 40.0 / cmax
    for _ in range(30):
        tb.step(1, dt)
        E.append(tb.energy())
    assert all(b <= a * (1 + 1e-13) for a, b in zip(E, E[1:])), E


def test_sh_plane_wave_transmission_and_reflection():
    """Block "-": x in [0, 1000] m, rho 2000, vs 2000; block "+": x in [1000, 2000] m, rho 2500,
    vs 3000 (Z2 / Z1 = 1.875).  A right-going SH pulse (v_z, sigma_xz = -Z1 v_z) starts at
    x = 600 m; faces normal to y are free (the wave satisfies them exactly), the faces normal to z
    are 2 km from the observation line, farther than any wave travels before the last sample."""
    from paper_2011_02600_gb300.multiblock import TwoBlockSolver
    order, h = 6, 10.0
    Lx, Ly, Lz = 1000.0, 150.0, 4000.0
    nm = (int(Lx / h) + 1, 16, int(Lz / 20.0) + 1)
    npl = nm
    rho1, vs1, rho2, vs2 = 2000.0, 2000.0, 2500.0, 3000.0
    Z1, Z2 = rho1 * vs1, rho2 * vs2

    def coords(x0, nodes):
        nq, nr, ns = nodes
        q = (np.arange(nq) / (nq - 1))[None, None, :]
        r = (np.arange(nr) / (nr - 1))[None, :, None]
        s = (np.arange(ns) / (ns - 1))[:, None, None]
        return np.stack([np.broadcast_to(c, (ns, nr, nq)) for c in (x0 + Lx * q, Ly * r + 0 * q, -Lz + Lz * s + 0 * q)])

    def medium(rho, vs, nodes):
        vp = math.sqrt(3.0) * vs
        mu = rho * vs * vs
        lam = rho * vp * vp - 2 * mu
        shape = (nodes[2], nodes[1], nodes[0])
        return np.stack([np.full(shape, rho), np.full(shape, lam), np.full(shape, mu)])
    Xm, Xp = coords(0.0, nm), coords(Lx, npl)
    bc = [("char", 0.0), ("char", 0.0), ("free",), ("free",), ("char", 0.0), ("char", 0.0)]
    tb = TwoBlockSolver(nm, npl, order, 64, bc, bc, xi=0)
    tb.setup(torch.from_numpy(Xm), torch.from_numpy(medium(rho1, vs1, nm)),
             torch.from_numpy(Xp), torch.from_numpy(medium(rho2, vs2, npl)))
    width, x0 = 40.0, 600.0
    Q = np.zeros((9,) + Xm.shape[1:])
    Q[2] = np.exp(-((Xm[0] - x0) / width) ** 2)
    Q[7] = -Z1 * Q[2]
    tb.m.set_state(torch.from_numpy(Q))
    tb.p.set_state(torch.zeros((9,) + Xp.shape[1:], dtype=torch.float64))
    dt = 0.4 * h / (math.sqrt(3.0) * vs2)
    t_end = (1000.0 - x0) / vs1 + 250.0 / vs2           # the transmitted pulse has gone 250 m on
    n = int(round(t_end / dt))
    tb.step(n, dt)
    kc, jc = nm[2] // 2, nm[1] // 2
    vm = tb.m.state()[2, kc, jc].cpu().numpy()
    vp_ = tb.p.state()[2, kc, jc].cpu().numpy()
    t = n * dt
    x = Xm[0, kc, jc]
    # reflected pulse in "-": centred at 1000 - vs1 (t - 0.2); transmitted in "+": at 1000 + vs2 (t - 0.2)
    t_hit = (1000.0 - x0) / vs1
    xr, xt = 1000.0 - vs1 * (t - t_hit), 1000.0 + vs2 * (t - t_hit)
    R, T = (Z1 - Z2) / (Z1 + Z2), 2 * Z1 / (Z1 + Z2)
    # pulse areas (the grid's trapezoidal sums of smooth pulses): the reflected pulse keeps the
    # incident width, the transmitted one is stretched by vs2 / vs1
    inc = math.sqrt(math.pi) * width
    wr = np.abs(x - xr) < 4 * width
    wt = np.abs(Xp[0, kc, jc] - xt) < 4 * width * vs2 / vs1
    area_r = float(np.sum(vm[wr])) * h
    area_t = float(np.sum(vp_[wt])) * h
    assert abs(area_r / inc - R) < 0.01 * abs(R), (area_r / inc, R)
    assert abs(area_t / (inc * vs2 / vs1) - T) < 0.01 * T, (area_t / (inc * vs2 / vs1), T)
