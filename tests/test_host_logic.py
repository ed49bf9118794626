"""CPU tests of the package's host-side helpers (no GPU): the double-couple moment tensor the
solver's sources are given, and the surrogate's parameter box."""
import math

import numpy as np

from oracle.source import moment_tensor
from paper_2011_02600_gb300 import surrogate as S
from paper_2011_02600_gb300.source_util import moment_tensor_voigt


def test_moment_tensor_matches_the_oracle():
    """The product's double couple (Sec. 7.1, Eq. momententor_pointsource) against the oracle's,
    written separately, over random fault angles and moments."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        st, dp, rk = rng.uniform(0, 2 * math.pi), rng.uniform(0.0, math.pi / 2), rng.uniform(-math.pi, math.pi)
        M0 = 10.0 ** rng.uniform(12, 18)
        got = np.array(moment_tensor_voigt(st, dp, rk, M0))
        assert np.allclose(got, moment_tensor(st, dp, rk, M0), rtol=0, atol=1e-13 * M0)


def test_moment_tensor_is_a_double_couple():
    """Eigenvalues (-M0, 0, M0): trace-free, scalar moment M0."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        st, dp, rk = rng.uniform(0, 2 * math.pi), rng.uniform(0.05, math.pi / 2), rng.uniform(-math.pi, math.pi)
        m = moment_tensor_voigt(st, dp, rk, 3.0)
        M = np.array([[m[0], m[3], m[4]], [m[3], m[1], m[5]], [m[4], m[5], m[2]]])
        assert np.allclose(np.sort(np.linalg.eigvalsh(M)), [-3.0, 0.0, 3.0], atol=1e-12)


def test_pure_dip_slip_on_a_vertical_fault_striking_north():
    """Strike 0 (fault plane x = 0 in east-north-up), dip 90 degrees, rake 90 degrees: slip is
    vertical on a plane with normal along x, so only M_xz is non-zero, with magnitude M0."""
    m = moment_tensor_voigt(0.0, math.pi / 2, math.pi / 2, 1.0)
    assert np.allclose([m[0], m[1], m[2], m[3], m[5]], 0.0, atol=1e-15)
    assert abs(abs(m[4]) - 1.0) < 1e-15
    assert np.allclose(m, moment_tensor(0.0, math.pi / 2, math.pi / 2, 1.0), atol=1e-15)


def test_parameter_box_sampling_and_mask():
    P = S.sample_params(3, 500)
    assert P.shape == (500, 7)
    assert S.in_box(P).all()
    assert np.array_equal(P, S.sample_params(3, 500))          # seeded
    assert not np.array_equal(P, S.sample_params(4, 500))
    lo, hi = np.asarray(S.PARAM_LO), np.asarray(S.PARAM_HI)
    # every coordinate fills its interval (uniform draws: min and max within 2 % of the ends)
    span = hi - lo
    assert np.all(P.min(axis=0) - lo < 0.02 * span) and np.all(hi - P.max(axis=0) < 0.02 * span)
    Q = P[:7].copy()
    for c in range(7):
        Q[c, c] = hi[c] + 1e-9 if c % 2 else lo[c] - 1e-9
    assert not S.in_box(Q).any()
    assert S.in_box(np.vstack([lo, hi])).all()                  # the box is closed
