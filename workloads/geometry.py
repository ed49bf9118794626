"""Boundary-conforming mesh maps x(q, r, s) for the synthetic workloads.

Every map takes reference coordinates q, r, s in [0, 1] (arrays that
broadcast against each other) and returns physical x, y, z in metres.  The
face s = 1 is the top (free) surface.  Arrays are laid out [s][r][q] when
built with ``node_coordinates``.
"""
import math

import numpy as np


def reference_axes(nodes, xp=np, dtype=None, device=None):
    """1D reference coordinates q_i = i/(n_q-1) etc. shaped for [s][r][q] broadcasting."""
    nq, nr, ns = nodes
    kw = {}
    if xp is not np:
        kw = dict(dtype=dtype, device=device)
    q = xp.arange(nq, **kw) / (nq - 1)
    r = xp.arange(nr, **kw) / (nr - 1)
    s = xp.arange(ns, **kw) / (ns - 1)
    return q.reshape(1, 1, nq), r.reshape(1, nr, 1), s.reshape(ns, 1, 1)


def topo_sinusoid_params(seed, n_modes=8, amp=600.0, extent=(60000.0, 60000.0)):
    """Seeded amplitudes, wavenumbers and phases of the sum-of-sinusoids top surface.

    sum |a_k| = amp; wavelengths between 3 km and 20 km; isotropic directions.
    """
    rng = np.random.default_rng([seed, 1001])
    a = rng.uniform(0.2, 1.0, n_modes)
    a *= amp / np.abs(a).sum()
    a *= rng.choice([-1.0, 1.0], n_modes)
    lam = rng.uniform(3000.0, 20000.0, n_modes)
    th = rng.uniform(0.0, 2 * math.pi, n_modes)
    kx = 2 * math.pi / lam * np.cos(th)
    ky = 2 * math.pi / lam * np.sin(th)
    ph = rng.uniform(0.0, 2 * math.pi, n_modes)
    return a, kx, ky, ph


def make_map(cfg_or_name, extent=None, xp=np, **params):
    """Return f(q, r, s) -> (x, y, z) for a named geometry."""
    if hasattr(cfg_or_name, "geometry"):
        name, extent = cfg_or_name.geometry, cfg_or_name.extent
        params = {**cfg_or_name.extra, "seed": cfg_or_name.seed, **params}
    else:
        name = cfg_or_name
    Lx, Ly, Lz = extent

    if name == "identity":
        def fmap(q, r, s):
            return Lx * q + 0 * r + 0 * s, Ly * r + 0 * q + 0 * s, -Lz + Lz * s + 0 * q + 0 * r
        return fmap

    if name == "gaussian_hill":
        amp = params.get("hill_amp", 1500.0)
        sig = params.get("hill_sigma", 4000.0)

        def fmap(q, r, s):
            x = Lx * q + 0 * r + 0 * s
            y = Ly * r + 0 * q + 0 * s
            h = amp * xp.exp(-((Lx * q - Lx / 2) ** 2 + (Ly * r - Ly / 2) ** 2) / sig ** 2)
            z = -Lz + s * (Lz + h)
            return x, y, z
        return fmap

    if name == "sinusoids":
        a, kx, ky, ph = topo_sinusoid_params(params.get("seed", 0), params.get("topo_modes", 8),
                                             params.get("topo_amp", 600.0), (Lx, Ly))

        def fmap(q, r, s):
            x = Lx * q + 0 * r + 0 * s
            y = Ly * r + 0 * q + 0 * s
            top = 0 * q + 0 * r
            for m in range(len(a)):
                top = top + float(a[m]) * xp.sin(float(kx[m]) * (Lx * q) + float(ky[m]) * (Ly * r) + float(ph[m]))
            z = -Lz + s * (Lz + top)
            return x, y, z
        return fmap

    if name == "curvy":
        # A fully curvilinear test map: every face curved, J > 0 for eps <= 0.1.
        eps = params.get("eps", 0.08)

        def fmap(q, r, s):
            x = Lx * (q + eps * xp.sin(math.pi * r + 0.3) * xp.cos(math.pi * s) + 0.5 * eps * q * r)
            y = Ly * (r + eps * xp.sin(math.pi * q + 0.5) * xp.sin(math.pi * s + 0.2))
            z = Lz * (s + eps * xp.sin(math.pi * q) * xp.cos(math.pi * r + 0.1) + 0.5 * eps * s * q)
            return x, y, z
        return fmap

    if name == "warped_interior":
        # Identity on every face, warped inside (boundary-conforming to a box).
        eps = params.get("eps", 0.05)

        def fmap(q, r, s):
            b = xp.sin(math.pi * q) * xp.sin(math.pi * r) * xp.sin(math.pi * s)
            return Lx * (q + eps * b), Ly * (r + 0.7 * eps * b), Lz * (s - 0.8 * eps * b)
        return fmap

    raise KeyError(name)


def node_coordinates(fmap, nodes, xp=np, dtype=None, device=None):
    """Physical coordinates of every node, arrays [s][r][q]."""
    q, r, s = reference_axes(nodes, xp, dtype, device)
    x, y, z = fmap(q, r, s)
    shape = (nodes[2], nodes[1], nodes[0])
    if xp is np:
        return tuple(np.broadcast_to(c, shape).copy() for c in (x, y, z))
    return tuple(c.expand(*shape).contiguous() for c in (x, y, z))


def coordinates_at(fmap, nodes, i, j, k):
    """Physical coordinates at node indices (i along q, j along r, k along s); numpy."""
    nq, nr, ns = nodes
    return fmap(np.asarray(i) / (nq - 1), np.asarray(j) / (nr - 1), np.asarray(k) / (ns - 1))
