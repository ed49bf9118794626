"""The adjoint workload: 129 x 129 x 97 nodes, Gaussian-hill top, order 4, 1500 steps, 64
surface receivers, true model = smooth background + 500 m Gaussian vs anomaly, gradient at the
background model.

* Full size, one source, FP64: the adjoint gradient agrees with central finite differences
  (two seeded smooth directions) to 1e-5.  FP32 forward with FP64 misfit: the gradient's
  directional derivatives stay within 1e-2 of the FP64 ones.
* Full size, the eight seeded sources as one batch, FP32: the batched gradient equals the sum
  of the eight single-source gradients (the members add into one FP64 gradient; only the order
  of those additions differs).
* The eight sources as one batch against central differences in the workload's 20 seeded
  directions, FP64, to 1e-5, on a 49 x 49 x 37 grid of the same workload over 300 steps: at full
  size the 40 batched FP64 forward runs would take about half an hour of GPU time.
"""
import pytest
import torch

from workloads.configs import config_by_name

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _direction(mats, seed, center_frac=(0.5, 0.5, 0.8), width=6.0):
    rho = mats[0]
    ns, nr, nq = rho.shape
    g = torch.Generator(device="cpu").manual_seed(seed)
    k = torch.arange(ns, dtype=torch.float64).view(ns, 1, 1)
    j = torch.arange(nr, dtype=torch.float64).view(1, nr, 1)
    i = torch.arange(nq, dtype=torch.float64).view(1, 1, nq)
    c = [center_frac[2] * (ns - 1), center_frac[1] * (nr - 1), center_frac[0] * (nq - 1)]
    shift = torch.randn(3, generator=g) * 3.0
    blob = torch.exp(-((k - c[0] - shift[0]) ** 2 + (j - c[1] - shift[1]) ** 2 + (i - c[2] - shift[2]) ** 2)
                     / (2 * width ** 2))
    w = torch.rand(3, generator=g) + 0.5
    return tuple((w[f] * blob).to(rho.device) * mats[f] for f in range(3))


def _dot(g, dm):
    return float(sum((g[f] * dm[f]).sum() for f in range(3)))


def test_workload4_gradient_full_size():
    from paper_2011_02600_gb300.adjoint import workload_problem
    cfg = config_by_name("adjoint129_o4")
    p64, true_m, back_m = workload_problem(cfg, 64)
    phi = p64.forward()
    assert phi > 0
    g64 = p64.gradient()
    dirs = [_direction(back_m, 1), _direction(back_m, 2)]
    h = 1e-5
    for dm in dirs:
        p64.set_material(*(m + h * d for m, d in zip(back_m, dm)))
        fp = p64.forward()
        p64.set_material(*(m - h * d for m, d in zip(back_m, dm)))
        fm = p64.forward()
        fd = (fp - fm) / (2 * h)
        got = _dot(g64, dm)
        assert abs(got - fd) < 1e-5 * abs(fd), (got, fd)
    del p64
    torch.cuda.empty_cache()
    p32, _, _ = workload_problem(cfg, 32)
    phi32 = p32.forward()
    g32 = p32.gradient()
    assert abs(phi32 - phi) < 1e-3 * phi
    for dm in dirs:
        assert abs(_dot(g32, dm) - _dot(g64, dm)) < 1e-2 * abs(_dot(g64, dm))


def test_workload4_all_sources_batched_full_size_fp32():
    from paper_2011_02600_gb300.adjoint import workload_problem
    cfg = config_by_name("adjoint129_o4")
    pb, _, _ = workload_problem(cfg, 32, source_index="all")
    assert pb.B == 8
    phi_b = pb.forward()
    g_b = pb.gradient()
    del pb
    torch.cuda.empty_cache()
    phi_s, g_s = 0.0, 0.0
    for m in range(8):
        p, _, _ = workload_problem(cfg, 32, source_index=m)
        phi_s += p.forward()
        g_s = g_s + p.gradient()
        del p
        torch.cuda.empty_cache()
    assert abs(phi_b - phi_s) < 1e-12 * phi_s
    for f in range(3):
        assert float((g_b[f] - g_s[f]).abs().max()) < 1e-10 * float(g_s[f].abs().max()), f


def test_workload4_all_sources_20_directions_fp64_reduced_grid():
    from paper_2011_02600_gb300.adjoint import workload_problem
    cfg = config_by_name("adjoint129_o4")
    pb, _, back_m = workload_problem(cfg, 64, source_index="all", nodes=(49, 49, 37), nsteps=300)
    pb.forward()
    g = pb.gradient()
    h = 1e-5
    worst = 0.0
    for seed in range(cfg.extra["n_fd_directions"]):
        dm = _direction(back_m, 100 + seed, width=3.0)
        pb.set_material(*(m + h * d for m, d in zip(back_m, dm)))
        fp = pb.forward()
        pb.set_material(*(m - h * d for m, d in zip(back_m, dm)))
        fm = pb.forward()
        fd = (fp - fm) / (2 * h)
        worst = max(worst, abs(_dot(g, dm) - fd) / abs(fd))
    assert worst < 1e-5, worst
