"""Time-step rule of the workloads (the paper does not state one).

dt = cfl * h_min / c_p,max, h_min the smallest distance between neighbouring
nodes along any grid line, c_p,max the largest P-wave speed.  The same dt is
handed to the oracle and to the CUDA path.
"""
import numpy as np


def stable_dt(x, y, z, rho, lam, mu, cfl):
    X = np.stack([np.asarray(c, dtype=float) for c in (x, y, z)])
    hmin = np.inf
    for ax in (1, 2, 3):
        d = np.diff(X, axis=ax)
        hmin = min(hmin, float(np.sqrt((d ** 2).sum(0)).min()))
    cp = float(np.sqrt((np.asarray(lam) + 2 * np.asarray(mu)) / np.asarray(rho)).max())
    return cfl * hmin / cp
