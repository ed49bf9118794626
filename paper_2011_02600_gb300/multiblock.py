"""Two curvilinear blocks on one device, coupled at a shared face by interface penalties.

Section 7.1 splits the LOH1 domain at its material discontinuity into two blocks, discretises
each on its own mesh and couples them weakly with penalties.  Here block "-" has the shared face
at xi = 1 of axis xi, block "+" at xi = 0; the faces hold the same nodes in the same order.
Before every Runge-Kutta stage each block writes its face trace (velocity, traction, impedances:
sbp_interface_trace), then both blocks run the stage, each reading the other's trace in its
interface penalty (SBP_BC_INTERFACE, sbp_set_interface).  Every step runs in the library's
kernels; this module holds the buffers and the order of the calls.
"""
import torch

from . import _lib as L
from .solver import ElasticSolver, _stream


def _face_shape(nodes, xi):
    nq, nr, ns = nodes
    return (ns, nr) if xi == 0 else (ns, nq) if xi == 1 else (nr, nq)


class TwoBlockSolver:
    """nodes_m, nodes_p: (nq, nr, ns) of blocks "-" and "+"; bc_m, bc_p: their six face
    conditions (the shared faces are set to the interface kind here); xi: the axis of the
    shared face (0: q)."""

    def __init__(self, nodes_m, nodes_p, order, precision=32, bc_m=None, bc_p=None, xi=0, device="cuda",
                 operator="upwind", batch=1):
        bc_m = list(bc_m or [("free",)] * 6)
        bc_p = list(bc_p or [("free",)] * 6)
        if _face_shape(nodes_m, xi) != _face_shape(nodes_p, xi):
            raise ValueError("the shared faces must hold the same node counts")
        self.xi, self.fm, self.fp = xi, 2 * xi + 1, 2 * xi
        bc_m[self.fm] = ("interface",)
        bc_p[self.fp] = ("interface",)
        kw = dict(device=device, operator=operator, batch=batch)
        self.m = ElasticSolver(nodes_m, order, precision, bc_m, **kw)
        self.p = ElasticSolver(nodes_p, order, precision, bc_p, **kw)
        nf = _face_shape(nodes_m, xi)[0] * _face_shape(nodes_m, xi)[1]
        self.tm = torch.zeros(8 * batch * nf, dtype=self.m.dtype, device=self.m.device)   # "-"'s trace
        self.tp = torch.zeros(8 * batch * nf, dtype=self.m.dtype, device=self.m.device)   # "+"'s trace
        L.sbp_set_interface(self.m.h, self.fm, self.tp)
        L.sbp_set_interface(self.p.h, self.fp, self.tm)
        self.t, self.nstep = 0.0, 0

    def setup(self, xyz_m, rlm_m, xyz_p, rlm_p, keep_metrics=False):
        self.m.setup(xyz_m, rlm_m, keep_metrics)
        self.p.setup(xyz_p, rlm_p, keep_metrics)

    def traces(self, qm=None, qp=None):
        """Both blocks' face traces, of the given states (flat buffers in the blocks' layouts) or
        of the current ones."""
        st = _stream()
        L.sbp_interface_trace(self.m.h, self.fm, qm, self.tm, st)
        L.sbp_interface_trace(self.p.h, self.fp, qp, self.tp, st)

    def rhs(self, Qm, Qp):
        """dQ/dt of both blocks for the states Qm, Qp ((9, ns, nr, nq) each)."""
        qm = self.m.to_layout(torch.as_tensor(Qm), self.m.dtype)
        qp = self.p.to_layout(torch.as_tensor(Qp), self.p.dtype)
        self.traces(qm, qp)
        om, op = self.m.new_fields(9), self.p.new_fields(9)
        L.sbp_rhs(self.m.h, qm, om, _stream())
        L.sbp_rhs(self.p.h, qp, op, _stream())
        return self.m.view(om, 9), self.p.view(op, 9)

    def stage(self, k, dt):
        self.traces()
        self.m.rk_stage(k, dt)
        self.p.rk_stage(k, dt)

    def step(self, n, dt):
        for _ in range(n):
            for k in range(5):
                self.stage(k, dt)
            self.t += dt
            self.nstep += 1
            self.m.set_time(self.t, self.nstep)
            self.p.set_time(self.t, self.nstep)

    def energy(self):
        """The discrete energy of the coupled system: the sum of the blocks' energies."""
        return self.m.energy() + self.p.energy()
