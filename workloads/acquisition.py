"""Seeded sources and surface receivers for the workloads.

Sources are given in reference coordinates (q, r, s) of the block with seeded
double-couple angles and moment; receivers are node indices on the top face.
"""
import math

import numpy as np


def surface_receivers(nodes, n_side, margin=0.2):
    """n_side x n_side receivers on the top face (s = 1), evenly spread inside a margin."""
    nq, nr, ns = nodes
    qs = np.linspace(margin, 1 - margin, n_side)
    out = []
    for r in qs:
        for q in qs:
            out.append((int(round(q * (nq - 1))), int(round(r * (nr - 1))), ns - 1))
    return out


def moment_sources(seed, n, M0=1.0e15, s_range=(0.67, 0.85), qr_range=(0.3, 0.7)):
    """n seeded point sources: reference position, strike, dip, rake (radians), moment."""
    rng = np.random.default_rng([seed, 5005])
    out = []
    for _ in range(n):
        out.append(dict(ref=(float(rng.uniform(*qr_range)), float(rng.uniform(*qr_range)), float(rng.uniform(*s_range))),
                        strike=float(rng.uniform(0, 2 * math.pi)), dip=float(rng.uniform(0.2, math.pi / 2)),
                        rake=float(rng.uniform(-math.pi, math.pi)), M0=M0))
    return out
