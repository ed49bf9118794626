"""The synthetic input recipes (CPU): each generator produces the statistics and values the
workloads state (media, topography, sources, receivers)."""
import math

import numpy as np

from workloads.acquisition import moment_sources, surface_receivers
from workloads.configs import config_by_name
from workloads.geometry import make_map, topo_sinusoid_params
from workloads.media import make_medium, vonkarman_modes


def test_vonkarman_perturbation_has_the_stated_rms():
    """delta = sum_m A cos(k_m . x + phi_m) with A = rms sqrt(2/M): its mean square over space
    is M A^2 / 2 = rms^2 (5 %); sampled over a large block it lands within a few percent."""
    cfg = config_by_name("topo1025_o6_fp32")
    k, phi, A = vonkarman_modes(cfg.seed, cfg.extra["vk_modes"], cfg.extra["vk_corr"], cfg.extra["vk_hurst"],
                                cfg.extra["vk_rms"])
    assert abs(A * math.sqrt(len(phi) / 2) - 0.05) < 1e-12
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 60000.0, (3, 40000))
    delta = sum(A * np.cos(k[m] @ x + phi[m]) for m in range(len(phi)))
    assert abs(np.sqrt(np.mean(delta ** 2)) - 0.05) < 0.005
    # wavenumbers around the correlation length (500 m), below the 100 m cut-off
    kmag = np.linalg.norm(k, axis=1)
    assert kmag.max() <= 2 * math.pi / 100.0 + 1e-12
    assert 0.3 < np.median(kmag) * 500.0 < 30.0


def test_gradient_vonkarman_medium_values():
    cfg = config_by_name("topo1025_o6_fp32")
    f = make_medium(cfg)
    z = np.array([0.0, -12000.0, -24000.0])
    rho, lam, mu = f(np.full(3, 30000.0), np.full(3, 30000.0), z)
    vs = np.sqrt(mu / rho)
    vp = np.sqrt((lam + 2 * mu) / rho)
    assert np.allclose(rho, [2200.0, 2550.0, 2900.0])
    assert np.allclose(vp / vs, math.sqrt(3.0))
    assert np.all(np.abs(vs / np.array([2000.0, 3000.0, 4000.0]) - 1) < 0.25)   # gradient x (1 + delta)


def test_sinusoid_topography_amplitude_and_wavelengths():
    cfg = config_by_name("topo1025_o6_fp32")
    a, kx, ky, ph = topo_sinusoid_params(cfg.seed, cfg.extra["topo_modes"], cfg.extra["topo_amp"], cfg.extent[:2])
    assert len(a) == 8 and abs(np.abs(a).sum() - 600.0) < 1e-9
    lam = 2 * math.pi / np.hypot(kx, ky)
    assert np.all((lam >= 3000.0) & (lam <= 20000.0))
    f = make_map(cfg)
    q, r = np.meshgrid(np.linspace(0, 1, 201), np.linspace(0, 1, 201))
    _, _, ztop = f(q, r, np.ones_like(q))
    _, _, zbot = f(q, r, np.zeros_like(q))
    assert np.abs(ztop).max() <= 600.0 + 1e-9 and np.abs(ztop).max() > 100.0
    assert np.allclose(zbot, -24000.0)


def test_layered_medium_and_gaussian_hill():
    cfg = config_by_name("hill129_o6")
    f = make_medium(cfg)
    rho, lam, mu = f(np.zeros(3), np.zeros(3), np.array([-500.0, -3000.0, -8000.0]))
    vs = np.sqrt(mu / rho)
    assert np.allclose(vs, [1000.0, 2000.0, 3500.0]) and np.allclose(rho, [2000.0, 2400.0, 2700.0])
    assert np.allclose(np.sqrt((lam + 2 * mu) / rho), math.sqrt(3.0) * vs)
    fm = make_map(cfg)
    _, _, zc = fm(np.array(0.5), np.array(0.5), np.array(1.0))
    _, _, zcorner = fm(np.array(0.0), np.array(0.0), np.array(1.0))
    _, _, zb = fm(np.array(0.3), np.array(0.7), np.array(0.0))
    assert abs(zc - 1500.0) < 1e-9                                    # summit of the hill
    assert abs(zcorner - 1500.0 * math.exp(-2 * 10000.0 ** 2 / 4000.0 ** 2)) < 1e-9
    assert abs(zb + 15000.0) < 1e-9


def test_sources_and_receivers():
    a = moment_sources(0, 8)
    b = moment_sources(0, 8)
    assert a == b and len(a) == 8                                     # seeded, reproducible
    for sp in a:
        q, r, s = sp["ref"]
        assert 0.3 <= q <= 0.7 and 0.3 <= r <= 0.7 and 0.67 <= s <= 0.85
        assert 0 <= sp["strike"] < 2 * math.pi and 0.2 <= sp["dip"] <= math.pi / 2
        assert -math.pi <= sp["rake"] <= math.pi and sp["M0"] == 1.0e15
    rec = surface_receivers((129, 129, 97), 8)
    assert len(rec) == 64 and len(set(rec)) == 64
    assert all(k == 96 and 25 <= i <= 103 and 25 <= j <= 103 for i, j, k in rec)
