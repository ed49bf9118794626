"""Seeded states Q = (vx, vy, vz, sxx, syy, szz, sxy, sxz, syz) for tests and runs.

Field order follows Section 2.1: velocities, then stresses in the order
(xx, yy, zz, xy, xz, yz).  Arrays are [9][s][r][q].
"""
import math

import numpy as np

FIELD_NAMES = ("vx", "vy", "vz", "sxx", "syy", "szz", "sxy", "sxz", "syz")


def random_state(nodes, seed, scale_v=1.0, scale_s=1.0e6):
    """I.i.d. normal state (numpy, FP64); small grids only."""
    nq, nr, ns = nodes
    rng = np.random.default_rng([seed, 3003])
    Q = rng.normal(size=(9, ns, nr, nq))
    Q[:3] *= scale_v
    Q[3:] *= scale_s
    return Q


def smooth_modes(seed, n_modes=4, kmax=5):
    """Per-field Fourier-mode parameters for ``smooth_state``."""
    rng = np.random.default_rng([seed, 4004])
    kap = rng.integers(-kmax, kmax + 1, size=(9, n_modes, 3)).astype(float)
    ph = rng.uniform(0, 2 * math.pi, size=(9, n_modes))
    amp = rng.uniform(0.5, 1.0, size=(9, n_modes))
    return kap, ph, amp


def smooth_state(nodes, seed, i, j, k, xp=np, scale_v=1.0, scale_s=1.0e6, n_modes=4):
    """Smooth random state at node indices (i, j, k) (arrays that broadcast).

    Field f = scale * sum_m amp sin(2 pi (k1 i/(nq-1) + k2 j/(nr-1) + k3 k/(ns-1)) + phase).
    Evaluable at any subset of nodes on either side.
    """
    nq, nr, ns = nodes
    kap, ph, amp = smooth_modes(seed, n_modes)
    qq, rr, ss = i / (nq - 1), j / (nr - 1), k / (ns - 1)
    out = []
    for f in range(9):
        acc = 0 * qq + 0 * rr + 0 * ss
        for m in range(n_modes):
            acc = acc + float(amp[f, m]) * xp.sin(2 * math.pi * (float(kap[f, m, 0]) * qq + float(kap[f, m, 1]) * rr
                                                                 + float(kap[f, m, 2]) * ss) + float(ph[f, m]))
        out.append(acc * (scale_v if f < 3 else scale_s))
    return out


def gaussian_pulse(x, y, z, center, width, xp=np):
    """Gaussian velocity pulse exp(-|x - c|^2 / (2 w^2)) on each velocity component; zero stress."""
    cx, cy, cz = center
    g = xp.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2.0 * width ** 2))
    zero = 0 * g
    return [g, g, g, zero, zero, zero, zero, zero, zero]
