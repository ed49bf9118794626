"""Elastic media (rho, lambda, mu) as closed-form functions of position.

All media are isotropic (Section 2.1): lambda = rho (vp^2 - 2 vs^2),
mu = rho vs^2.  Depth is d = -z (z = 0 is the flat reference level; the
topography rises above it).
"""
import math

import numpy as np


def lame(rho, vp, vs):
    mu = rho * vs ** 2
    lam = rho * vp ** 2 - 2.0 * mu
    return rho, lam, mu


def vonkarman_modes(seed, n_modes, corr, hurst, rms):
    """Random-mode (spectral sampling) representation of a von Karman random field.

    delta(x) = sum_m A cos(k_m . x + phi_m), A = rms * sqrt(2 / n_modes); |k_m| is
    drawn from the 3D radial density k^2 (1 + k^2 a^2)^-(hurst + 3/2), directions
    are isotropic.  Returns (k: [n_modes, 3], phi: [n_modes], A).
    """
    rng = np.random.default_rng([seed, 2002])
    kmax = 2 * math.pi / 100.0
    kk = np.linspace(0.0, kmax, 20001)
    dens = kk ** 2 * (1 + (kk * corr) ** 2) ** (-(hurst + 1.5))
    cdf = np.cumsum(dens)
    cdf /= cdf[-1]
    kmag = np.interp(rng.uniform(0, 1, n_modes), cdf, kk)
    u = rng.normal(size=(n_modes, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    k = u * kmag[:, None]
    phi = rng.uniform(0, 2 * math.pi, n_modes)
    return k, phi, rms * math.sqrt(2.0 / n_modes)


def make_medium(cfg_or_name, xp=np, **params):
    """Return f(x, y, z) -> (rho, lam, mu)."""
    if hasattr(cfg_or_name, "medium"):
        name = cfg_or_name.medium
        params = {**cfg_or_name.extra, "seed": cfg_or_name.seed, **params}
    else:
        name = cfg_or_name

    if name == "homogeneous":
        rho0 = params.get("rho", 2700.0)
        vp0 = params.get("vp", 6000.0)
        vs0 = params.get("vs", 3464.0)

        def fmed(x, y, z):
            one = 0 * x + 0 * y + 0 * z + 1.0
            return lame(rho0 * one, vp0 * one, vs0 * one)
        return fmed

    if name == "layered3":
        # Interfaces at 1 km and 5 km depth; vs 1.0/2.0/3.5 km/s, vp = sqrt(3) vs.
        def fmed(x, y, z):
            d = -z + 0 * x + 0 * y
            vs = xp.where(d < 1000.0, 1000.0 + 0 * d, xp.where(d < 5000.0, 2000.0 + 0 * d, 3500.0 + 0 * d))
            rho = xp.where(d < 1000.0, 2000.0 + 0 * d, xp.where(d < 5000.0, 2400.0 + 0 * d, 2700.0 + 0 * d))
            return lame(rho, math.sqrt(3.0) * vs, vs)
        return fmed

    if name == "smooth_gradient":
        # Smooth depth gradient (used where a differentiable medium is wanted).
        Lz = params.get("Lz", 15000.0)

        def fmed(x, y, z):
            t = xp.clip((-z + 0 * x + 0 * y) / Lz, 0.0, 1.0)
            vs = 1500.0 + 2000.0 * t
            rho = 2200.0 + 500.0 * t
            return lame(rho, math.sqrt(3.0) * vs, vs)
        return fmed

    if name in ("smooth_background", "smooth_anomaly"):
        # Smooth depth gradient over the block (vs 1.5 -> 3.5 km/s, rho 2200 -> 2700, vp = sqrt(3) vs);
        # "smooth_anomaly" multiplies vs by 1 + a exp(-|x - x0|^2 / (2 r^2)) (a Gaussian vs anomaly).
        Lz = params.get("Lz", 15000.0)
        x0 = params.get("anomaly_center", (10000.0, 10000.0, -3000.0))
        rad = params.get("anomaly_radius", 500.0)
        amp = params.get("anomaly_amp", 0.1) if name == "smooth_anomaly" else 0.0

        def fmed(x, y, z):
            t = xp.clip(-z / Lz + 0 * x + 0 * y, 0.0, 1.0)
            vs = 1500.0 + 2000.0 * t
            rho = 2200.0 + 500.0 * t
            if amp:
                g = xp.exp(-((x - x0[0]) ** 2 + (y - x0[1]) ** 2 + (z - x0[2]) ** 2) / (2.0 * rad ** 2))
                vs = vs * (1.0 + amp * g)
            return lame(rho, math.sqrt(3.0) * vs, vs)
        return fmed

    if name == "gradient_vonkarman":
        Lz = params.get("Lz", 24000.0)
        k, phi, A = vonkarman_modes(params.get("seed", 0), params.get("vk_modes", 64),
                                    params.get("vk_corr", 500.0), params.get("vk_hurst", 0.5),
                                    params.get("vk_rms", 0.05))

        def fmed(x, y, z):
            t = xp.clip(-z / Lz + 0 * x + 0 * y, 0.0, 1.0)
            vs0 = 2000.0 + 2000.0 * t
            rho = 2200.0 + 700.0 * t
            delta = 0 * t
            for m in range(len(phi)):
                delta = delta + A * xp.cos(float(k[m, 0]) * x + float(k[m, 1]) * y + float(k[m, 2]) * z + float(phi[m]))
            vs = vs0 * (1.0 + delta)
            return lame(rho, math.sqrt(3.0) * vs, vs)
        return fmed

    raise KeyError(name)
