"""Receiver misfit and its material gradient by the discrete adjoint (torch autograd).

The forward run is the library's fused Runge-Kutta stepping; the misfit
Phi = sum_n 1/2 dt sum_r |v(x_r, t_{n+1}) - d_r,n|^2 is accumulated in FP64 by
the misfit kernel.  The gradient with respect to rho, lambda and mu at every
node comes from the exact adjoint of each fused stage (``sbp_adjoint_stage``)
run backwards in time.  States are checkpointed every C = ceil(sqrt(N)) steps
in the forward run; in the backward run each segment is recomputed from its
checkpoint, and each step's five stage inputs are recomputed from the step's
state before its adjoint stages run.
"""
import math

import torch

from . import _lib as L
from .solver import _stream


class MisfitProblem:
    """solver: ElasticSolver set up with keep_metrics=True; receivers: (i, j, k) list;
    data: FP64 tensor [n_rec][3][nsteps], or [B][n_rec][3][nsteps] for a batched solver of B
    states; source: dict for ElasticSolver.set_source or None; sources: for a batched solver,
    one dict (ref, moment) per state, sharing the Ricker frequency f0.  The misfit is the sum
    over the states; the gradient, that of the sum (the adjoint stages run every state in one
    launch and add into one gradient)."""

    def __init__(self, solver, receivers, data, dt, nsteps, source=None, checkpoint_every=None, sources=None,
                 f0=2.0):
        if solver.jmet is None:
            raise ValueError("the solver must keep its metrics (setup(..., keep_metrics=True))")
        self.s = solver
        self.receivers = [tuple(int(x) for x in r) for r in receivers]
        self.nsteps = int(nsteps)
        self.dt = float(dt)
        self.B = solver.batch
        self.data = self._layout(data)
        self.C = int(checkpoint_every or max(1, math.ceil(math.sqrt(self.nsteps))))
        self.source = source
        s = solver
        self.rlmj = s.new_fields(4, torch.float64)
        self.acc = torch.zeros(self.B * len(self.receivers) * 3, dtype=torch.float64, device=s.device)
        s.set_receivers(self.receivers, max(1, self.nsteps))
        if sources is not None:
            s.set_sources(sources, f0=f0)
        elif source is not None:
            s.set_source(**source)
        self.ckpt = {}
        # one sbp_adjoint_step per step (the stages' pointwise preps fused into the L^T passes);
        # False: sbp_adjoint_stage five times
        self.fused = True

    def _layout(self, data):
        """[nsteps][B * n_rec * 3] (member-major, as the misfit kernel reads it)."""
        d = torch.as_tensor(data, dtype=torch.float64, device=self.s.device)
        if d.dim() == 3:
            d = d.unsqueeze(0)
        return d.permute(3, 0, 1, 2).reshape(d.shape[3], -1).contiguous()

    def recorded(self):
        """The traces of the last forward run as data: [B][n_rec][3][nsteps] (FP64)."""
        n_rec = len(self.receivers)
        return self.s.traces.view(self.B, -1, 3, max(1, self.nsteps))[:, :n_rec].double()

    def set_material(self, rho, lam, mu):
        s = self.s
        rlm = s.new_fields(3, torch.float64)
        v = s.view(rlm, 3)
        for f, m in enumerate((rho, lam, mu)):
            v[f].copy_(torch.as_tensor(m, dtype=torch.float64))
        L.sbp_set_material(s.h, s.jmet, rlm, _stream())
        r = s.view(self.rlmj, 4)
        r[:3].copy_(v)
        r[3].copy_(s.view(s.jmet, 10)[0])
        bits = s.status()
        if bits & 6:
            raise L.SbpError(6, f"material check failed (status {bits})")

    def _reset(self):
        s = self.s
        for b in s.qbuf:
            b.zero_()
        s.dq.zero_()
        s.set_time(0.0, 0)

    def forward(self):
        """Run the forward problem from rest; returns Phi (float) and keeps checkpoints."""
        s = self.s
        self._reset()
        self.acc.zero_()
        self.ckpt = {0: s.qbuf[s.current].clone()}
        st = _stream()
        for n in range(self.nsteps):
            L.sbp_step_n(s.h, 1, self.dt, st)
            L.sbp_misfit(s.h, s.qbuf[s.current], self.data[n], self.dt, self.acc, None, st)
            if (n + 1) % self.C == 0 and n + 1 < self.nsteps:
                self.ckpt[n + 1] = s.qbuf[s.current].clone()
        return float(self.acc.sum())

    def _load(self, q, n):
        s = self.s
        s.qbuf[s.current].copy_(q)
        s.set_time(n * self.dt, n)

    def gradient(self):
        """d Phi / d(rho, lambda, mu): FP64 tensor [3][ns][nr][nq] (after forward())."""
        s = self.s
        st = _stream()
        nf = 9 * self.B
        ubar = s.new_fields(nf)
        wbar = s.new_fields(nf)
        scratch = s.new_fields(2 * nf)
        grad = s.new_fields(3, torch.float64)
        stages = s.new_fields(5 * nf)          # U_0..U_4 back to back
        g = nf * s.fs
        stage_in = [stages[k * g:(k + 1) * g] for k in range(5)]
        starts = sorted(self.ckpt)
        for seg in reversed(starts):
            end = min(seg + self.C, self.nsteps)
            states = [self.ckpt[seg]]
            self._load(self.ckpt[seg], seg)
            for n in range(seg, end):
                L.sbp_step_n(s.h, 1, self.dt, st)
                states.append(s.qbuf[s.current].clone())
            for n in reversed(range(seg, end)):
                L.sbp_misfit(s.h, states[n + 1 - seg], self.data[n], self.dt, None, ubar, st)
                self._load(states[n - seg], n)
                for k in range(5):
                    stage_in[k].copy_(s.qbuf[s.current])
                    L.sbp_rk_stage(s.h, k, self.dt, st)
                wbar.zero_()
                if self.fused:
                    L.sbp_adjoint_step(s.h, self.dt, stages, ubar, wbar, scratch, self.rlmj, grad, st)
                else:
                    for k in reversed(range(5)):
                        L.sbp_adjoint_stage(s.h, k, self.dt, stage_in[k], ubar, wbar, scratch, self.rlmj, grad,
                                            st)
            del states
        return s.view(grad, 3).clone()


class ElasticMisfit(torch.autograd.Function):
    """Phi(rho, lambda, mu) with the adjoint gradient as backward."""

    @staticmethod
    def forward(ctx, rho, lam, mu, problem):
        problem.set_material(rho, lam, mu)
        phi = problem.forward()
        ctx.problem = problem
        return torch.tensor(phi, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, g):
        grad = ctx.problem.gradient()
        return g * grad[0], g * grad[1], g * grad[2], None


def workload_materials(solver, cfg, anomaly):
    """(rho, lambda, mu) of the workload's background (anomaly=False) or true model, on the device."""
    from workloads.geometry import make_map, reference_axes
    from workloads.media import make_medium
    name = "smooth_anomaly" if anomaly else cfg.medium
    fmap = make_map(cfg, xp=torch)
    fmed = make_medium(name, xp=torch, **{**cfg.extra, "seed": cfg.seed})
    q, r, s = reference_axes(cfg.nodes, torch, torch.float64, solver.device)
    x, y, z = fmap(q, r, s)
    shape = (cfg.nodes[2], cfg.nodes[1], cfg.nodes[0])
    return tuple(m.expand(*shape).contiguous() for m in fmed(x, y, z))


def workload_problem(cfg, precision, source_index=0, nsteps=None, checkpoint_every=None, nodes=None):
    """MisfitProblem for the adjoint workload: data recorded with the true model (background
    plus a Gaussian vs anomaly) at the 64 surface receivers for one of its seeded sources
    (source_index), or for all of them as one batch (source_index = "all": the workload's
    eight sources, one state each); material set to the background.  nodes: a smaller grid of
    the same workload (tests).  Returns (problem, true_material, background_material)."""
    import dataclasses
    from workloads.acquisition import moment_sources, surface_receivers
    from .workload_setup import build_solver
    from .source_util import moment_tensor_voigt
    if nodes is not None:
        cfg = dataclasses.replace(cfg, nodes=tuple(nodes))
    nsteps = nsteps or cfg.steps
    srcs = moment_sources(cfg.seed, cfg.extra.get("n_sources", 8))
    chosen = srcs if source_index == "all" else [srcs[source_index]]
    s, info = build_solver(cfg, precision=precision, keep_metrics=True, batch=len(chosen))
    sources = [dict(ref=sp["ref"], moment=list(moment_tensor_voigt(sp["strike"], sp["dip"], sp["rake"], sp["M0"])))
               for sp in chosen]
    rec = surface_receivers(cfg.nodes, 8)
    n_rec = len(rec)
    f0 = cfg.extra.get("f0", 2.0)
    zeros = torch.zeros(len(chosen), n_rec, 3, nsteps, dtype=torch.float64)
    if len(chosen) == 1:
        p = MisfitProblem(s, rec, zeros[0], info["dt"], nsteps, checkpoint_every=checkpoint_every,
                          source=dict(**sources[0], stf="ricker", f0=f0))
    else:
        p = MisfitProblem(s, rec, zeros, info["dt"], nsteps, checkpoint_every=checkpoint_every, sources=sources,
                          f0=f0)
    true_m = workload_materials(s, cfg, anomaly=True)
    back_m = workload_materials(s, cfg, anomaly=False)
    p.set_material(*true_m)
    p.forward()
    p.data = p._layout(p.recorded())
    p.set_material(*back_m)
    return p, true_m, back_m
