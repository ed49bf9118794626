"""Set up an ElasticSolver for one of the synthetic workloads on the GPU.

Coordinates, media and initial states come from the seeded generators in
``workloads`` (closed-form functions evaluated with torch on the device, in
chunks of s-planes so that the FP64 temporaries stay small); the metrics,
coefficients and every later step run in the library's kernels.
"""
import math

import torch

from workloads.geometry import make_map
from workloads.media import make_medium

from .solver import ElasticSolver

CHUNK = 32


def _fill_chunks(s, buf, nf, fn):
    """buf (flat, layout of s) <- fn(q, r, s_plane_block) for blocks of s-planes."""
    nq, nr, ns = s.nodes
    v = s.view(buf, nf)
    dev = s.device
    q = (torch.arange(nq, device=dev, dtype=torch.float64) / (nq - 1)).view(1, 1, nq)
    r = (torch.arange(nr, device=dev, dtype=torch.float64) / (nr - 1)).view(1, nr, 1)
    for k0 in range(0, ns, CHUNK):
        k1 = min(ns, k0 + CHUNK)
        sp = (torch.arange(k0, k1, device=dev, dtype=torch.float64) / (ns - 1)).view(-1, 1, 1)
        vals = fn(q, r, sp)
        for f in range(nf):
            v[f, k0:k1].copy_(vals[f].expand(k1 - k0, nr, nq))


def build_solver(cfg, precision=None, device="cuda", keep_metrics=False, batch=1, operator="upwind"):
    """ElasticSolver for a WorkloadConfig with metrics and material set (operator: "upwind" or
    "traditional", of the config's order).

    Returns (solver, info) with info = dict(dt=..., hmin=..., cpmax=...)."""
    precision = precision or cfg.precisions[0]
    s = ElasticSolver(cfg.nodes, cfg.order, precision, list(cfg.bc), device=device, batch=batch,
                      operator=operator)
    fmap = make_map(cfg, xp=torch)
    fmed = make_medium(cfg, xp=torch)
    import paper_2011_02600_gb300._lib as L
    from .solver import _stream
    xyz = s.new_fields(3, torch.float64)
    _fill_chunks(s, xyz, 3, lambda q, r, sp: fmap(q, r, sp))
    jmet = s.new_fields(10, torch.float64)
    L.sbp_metrics(s.h, xyz, jmet, _stream())
    rlm = s.new_fields(3, torch.float64)
    _fill_chunks(s, rlm, 3, lambda q, r, sp: fmed(*fmap(q, r, sp)))
    # time step: dt = cfl * h_min / c_p,max (the workloads' rule)
    X = s.view(xyz, 3)
    hmin = math.inf
    for ax in (1, 2, 3):
        for k0 in range(0, cfg.nodes[2], CHUNK):
            blk = X[:, k0:min(cfg.nodes[2], k0 + CHUNK + 1)]
            d = torch.diff(blk, dim=ax)
            if d.numel():
                hmin = min(hmin, float(torch.sqrt((d ** 2).sum(0)).min()))
    R = s.view(rlm, 3)
    cpmax = 0.0
    for k0 in range(0, cfg.nodes[2], CHUNK):
        blk = R[:, k0:k0 + CHUNK]
        cpmax = max(cpmax, float(torch.sqrt((blk[1] + 2 * blk[2]) / blk[0]).max()))
    del xyz
    L.sbp_set_material(s.h, jmet, rlm, _stream())
    del rlm
    bits = L.sbp_status(s.h, _stream())
    if bits & 6:
        raise L.SbpError(6, f"mesh/material check failed (status {bits})")
    s.jmet = jmet if keep_metrics else None
    del jmet
    torch.cuda.empty_cache()
    return s, dict(dt=cfg.cfl * hmin / cpmax, hmin=hmin, cpmax=cpmax)
