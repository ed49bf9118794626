"""Pins of the oracle's two-block interface coupling (oracle/multiblock.py).

* The interface Riemann problem (the hat variables): both outgoing characteristics are kept,
  velocity and traction are continuous, and for a wave arriving from one side onto a block at
  rest the transmitted and reflected velocity amplitudes are the textbook coefficients
  2 Z-/(Z- + Z+) and (Z- - Z+)/(Z- + Z+).
* Energy: with free surfaces on every outer face, <Q-, P~^-1 dQ-/dt>_H + <Q+, P~^-1 dQ+/dt>_H
  equals minus the penalties' dissipation I(sum |G|^2/Z) on the two interface faces (the hat
  terms I(vhat That) of the two sides cancel: the faces share nodes, normal and weights), so
  the coupled scheme is energy stable; random states, random media, curved blocks and interface.
* A state that is continuous across the interface in one medium draws no penalty.
* A planted mistake (a traction sign in the hat variables) breaks the energy identity."""
import numpy as np
import pytest

from oracle import multiblock as MB
from oracle.elastic import Scheme, inner_H
from oracle.metrics import metrics
from workloads.fields import random_state, smooth_state
from workloads.twoblock import block_coordinates, two_block_maps

FREE_M = [("free",), ("interface",), ("free",), ("free",), ("free",), ("free",)]
FREE_P = [("interface",), ("free",), ("free",), ("free",), ("free",), ("free",)]


def test_interface_hat_closed_forms():
    rng = np.random.default_rng(1)
    for _ in range(100):
        vm, Tm, vp, Tp = rng.normal(size=4)
        Zm, Zp = rng.uniform(0.5, 3.0, size=2)
        vh, Th = MB.interface_hat(vm, Tm, Zm, vp, Tp, Zp)
        assert abs((Zm * vh - Th) - (Zm * vm - Tm)) < 1e-13
        assert abs((Zp * vh + Th) - (Zp * vp + Tp)) < 1e-13
        # continuous fields are their own hat values
        vh2, Th2 = MB.interface_hat(vm, Tm, Zm, vm, Tm, Zp)
        assert abs(vh2 - vm) < 1e-13 and abs(Th2 - Tm) < 1e-13
    # a right-going wave in "-" (T = -Z- v, amplitude v_i) onto "+" at rest
    for Zm, Zp in [(1.0, 3.0), (2.5, 0.7), (1.3, 1.3)]:
        vi = 0.8
        vh, Th = MB.interface_hat(vi, -Zm * vi, Zm, 0.0, 0.0, Zp)
        assert abs(vh - 2 * Zm / (Zm + Zp) * vi) < 1e-14                 # transmitted
        assert abs((vh - vi) - (Zm - Zp) / (Zm + Zp) * vi) < 1e-14       # reflected


def _blocks(order, nodes_m=(13, 14, 15), nodes_p=(17, 14, 15), d=0.05, warp=0.2):
    fm, fp = two_block_maps(0.7, 1.1, 1.2, 0.9, d=d, warp=warp)
    Xm, Xp = block_coordinates(fm, nodes_m), block_coordinates(fp, nodes_p)
    assert np.array_equal(Xm[0][:, :, -1], Xp[0][:, :, 0]) and np.array_equal(Xm[2][:, :, -1], Xp[2][:, :, 0])
    Jm, am = metrics(*Xm, order)
    Jp, ap = metrics(*Xp, order)
    return Xm, Xp, Jm, am, Jp, ap, Scheme(order, nodes_m), Scheme(order, nodes_p)


def _medium(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(1.0, 2.0, shape), rng.uniform(0.2, 2.0, shape), rng.uniform(0.5, 1.5, shape)


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_two_block_energy_identity(order):
    nm, npl = (13, 14, 15), (17, 14, 15)
    nm = tuple(max(n, 16) for n in nm) if order >= 6 else nm
    npl = tuple(max(n, 16) for n in npl) if order >= 6 else npl
    Xm, Xp, Jm, am, Jp, ap, sm, sp = _blocks(order, nm, npl)
    mat_m, mat_p = _medium(Jm.shape, 4), _medium(Jp.shape, 5)
    Qm, Qp = random_state(nm, 8, 1.0, 1.0), random_state(npl, 9, 1.0, 1.0)
    lhs, want, diag = MB.interface_energy_rate(Qm, Qp, sm, sp, am, ap, mat_m, mat_p, FREE_M, FREE_P, 0)
    from oracle.elastic import surface_integral
    hat_m = surface_integral(diag["-"]["hat"], sm, 0, diag["-"]["anorm"])
    hat_p = surface_integral(diag["+"]["hat"], sp, 0, diag["+"]["anorm"])
    scale = abs(want)
    assert want < 0 and scale > 0
    assert abs(hat_m - hat_p) < 1e-12 * (abs(hat_m) + scale)
    assert abs(lhs - want) < 1e-11 * scale, (lhs, want)


def test_continuous_state_in_one_medium_draws_no_penalty():
    order = 4
    Xm, Xp, Jm, am, Jp, ap, sm, sp = _blocks(order)
    # one medium and one smooth state, both functions of position, evaluated on both blocks
    def medium(x, y, z):
        return 1.5 + 0.1 * np.sin(x), 1.0 + 0.2 * np.cos(y), 0.8 + 0.1 * np.sin(z)

    def state(x, y, z):
        return np.stack([np.sin(1.3 * x + 0.7 * y + c) * np.cos(0.9 * z - c) for c in range(9)])
    mat_m, mat_p = medium(*Xm), medium(*Xp)
    Qm, Qp = state(*Xm), state(*Xp)
    diag = {}
    MB.two_block_rhs_raw(Qm, Qp, sm, sp, am, ap, mat_m, mat_p, FREE_M, FREE_P, 0, diag)
    for side in "-+":
        assert max(np.abs(v).max() for v in diag[side]["sat_v"]) < 1e-12
        assert max(np.abs(e).max() for e in diag[side]["sat_e"]) < 1e-12


def test_planted_sign_mistake_breaks_the_identity(monkeypatch):
    order = 4
    Xm, Xp, Jm, am, Jp, ap, sm, sp = _blocks(order)
    mat_m, mat_p = _medium(Jm.shape, 4), _medium(Jp.shape, 5)
    Qm, Qp = random_state((13, 14, 15), 8, 1.0, 1.0), random_state((17, 14, 15), 9, 1.0, 1.0)
    good = MB.interface_hat

    def wrong(vm, Tm, Zm, vp, Tp, Zp):          # the "+" side's traction enters with the wrong sign
        return good(vm, Tm, Zm, vp, -Tp, Zp)
    monkeypatch.setattr(MB, "interface_hat", wrong)
    lhs, want, _ = MB.interface_energy_rate(Qm, Qp, sm, sp, am, ap, mat_m, mat_p, FREE_M, FREE_P, 0)
    assert abs(lhs - want) > 1e-6 * abs(want) or want > 0
