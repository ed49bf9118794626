"""The paper's operator comparisons on the Gaussian-hill workload, on the GPU.

Section 6.2 finds, from the numerical dispersion relations of Tables 1 and 2, that the even
upwind orders 2, 4, 6 carry no spurious unresolved wave modes while the odd upwind orders and the
traditional central operators do; Section 7.2 shows the same in seismograms on topography, each
scheme at one resolution against a solution on a twice finer mesh.  This module runs that
experiment on the synthetic curvilinear free-surface workload (129 x 129 x 97 nodes over
20 x 20 x 15 km, Gaussian hill, three layers, 2 Hz Ricker moment-tensor source 3 km below the
summit): every operator at the workload's resolution, one reference run at `refine` times finer
spacing, and the relative L2 error of the surface seismograms against the reference at the same
nodes and times.  Every step runs in the library's kernels.
"""
import dataclasses

import numpy as np
import torch

from workloads.acquisition import moment_sources
from workloads.configs import config_by_name

from .source_util import moment_tensor_voigt
from .workload_setup import build_solver

# (order, operator family) of Tables 1 and 2
OPERATORS = [(2, "upwind"), (3, "upwind"), (4, "upwind"), (5, "upwind"), (6, "upwind"), (7, "upwind"),
             (2, "traditional"), (4, "traditional"), (6, "traditional")]


def coarse_receivers(nodes, n_side=4, margin=0.2):
    """n_side x n_side surface nodes of the coarse grid, evenly spread inside a margin."""
    nq, nr, ns = nodes
    idx = [int(round((margin + (1 - 2 * margin) * a / (n_side - 1)) * (n - 1))) for n in (nq, nr)
           for a in range(n_side)]
    iq, ir = idx[:n_side], idx[n_side:]
    return [(i, j, ns - 1) for j in ir for i in iq]


def hill_run(order, operator, refine=1, precision=32, t_end=None, dt_coarse=None, f0=None, cfl=None,
             base="hill129_o6"):
    """One run of the Gaussian-hill workload with spacing h / refine.  The time step is
    dt_coarse / refine (dt_coarse: the workload's CFL rule on the coarse grid, at Courant number
    cfl, when None) and the run covers t_end (default: the workload's steps at dt_coarse); f0:
    the Ricker frequency (default the workload's).  Returns (traces [receiver][component][coarse
    sample], dt_coarse, seconds of GPU time): the velocity at the coarse receivers' nodes after
    every coarse step."""
    cfg = config_by_name(base)
    coarse = cfg.nodes
    nodes = tuple((n - 1) * refine + 1 for n in coarse)
    rc = dataclasses.replace(cfg, nodes=nodes, order=order, cfl=cfl or cfg.cfl)
    s, info = build_solver(rc, precision=precision, keep_metrics=True, operator=operator)
    if dt_coarse is None:
        if refine != 1:
            raise ValueError("pass dt_coarse for a refined run")
        dt_coarse = info["dt"]
    dt = dt_coarse / refine
    t_end = cfg.steps * dt_coarse if t_end is None else t_end
    n_coarse = int(round(t_end / dt_coarse))
    sp = moment_sources(cfg.seed, 1)[0]
    h = cfg.extra["hill_amp"]
    Lz = cfg.extent[2]
    s_ref = (Lz - cfg.extra["src_depth"] + h) / (Lz + h)          # 3 km below the summit
    s.set_source((0.5, 0.5, s_ref), moment_tensor_voigt(sp["strike"], sp["dip"], sp["rake"], sp["M0"]),
                 "ricker", f0=f0 or cfg.extra["f0"])
    rec = [(i * refine, j * refine, nodes[2] - 1) for (i, j, _) in coarse_receivers(coarse)]
    tr = s.set_receivers(rec, n_coarse * refine)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    s.step(n_coarse * refine, dt)
    ev[1].record()
    torch.cuda.synchronize()
    if s.status() != 0:
        raise RuntimeError(f"order {order} {operator}: device status {s.status()}")
    out = tr.double().cpu().numpy()[:, :, refine - 1::refine]   # after coarse steps 1..n_coarse
    del s
    torch.cuda.empty_cache()
    return out, dt_coarse, ev[0].elapsed_time(ev[1]) / 1e3


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


# The comparison's run: a 1 Hz Ricker source (the slowest layer, vs = 1 km/s, then has about
# 2.6 nodes per shortest significant S wavelength, 2.5 f0, on the 156 m grid: marginally
# resolved, the regime of Section 7.2), 12 s of simulated time, and one time step for every
# operator (as in Section 7.2), at Courant number 0.25: the upwind order-2 pair, whose D+ has
# the largest spectral radius, is unstable at the workload's 0.5.
COMPARE_F0 = 1.0
COMPARE_T_END = 12.0
COMPARE_CFL = 0.25


def compare(operators=OPERATORS, refine=2, ref_order=6, precision=32, t_end=COMPARE_T_END, f0=COMPARE_F0,
            cfl=COMPARE_CFL):
    """Relative L2 seismogram error of each operator against the refined reference run.
    Returns dict(errors={(order, family): err}, ref=(order, refine), dt=..., seconds=...)."""
    first, dt_c, t_first = hill_run(ref_order, "upwind", 1, precision, t_end, f0=f0, cfl=cfl)
    ref, _, t_ref = hill_run(ref_order, "upwind", refine, precision, t_end, dt_coarse=dt_c, f0=f0, cfl=cfl)
    errors, secs = {}, {"reference": t_ref}
    for order, fam in operators:
        if (order, fam) == (ref_order, "upwind"):
            tr, t = first, t_first
        else:
            tr, _, t = hill_run(order, fam, 1, precision, t_end, dt_coarse=dt_c, f0=f0, cfl=cfl)
        errors[(order, fam)] = rel_l2(tr, ref)
        secs[(order, fam)] = t
    return dict(errors=errors, ref=(ref_order, refine), dt=dt_c, seconds=secs, samples=ref.shape[-1], f0=f0,
                cfl=cfl, t_end=t_end)
