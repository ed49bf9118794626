"""One block decomposed along s into slabs, one per device, with the halo exchange.

The paper's own code splits its blocks over MPI ranks and exchanges ghost nodes of the
stencil's width at every stage (Section 7.2's scaling runs); here the block is cut into slabs of
s-planes (s is the slowest axis, so a slab's planes are contiguous in every field), each slab
lives on one device with `reach` ghost planes at each inner end (reach = max(r, q) of the
interior stencil: 4 for order 6), and after every Runge-Kutta stage each slab sends its first
and last `reach` owned planes of the 9 state fields to its neighbours, which store them as their
ghost planes.  The stage kernels compute the owned planes only, with closures and penalties at
the block's faces alone (sbp_set_slab), so the owned planes evolve exactly as in the undivided
block.

Transports: DistTransport (torch.distributed point-to-point: NCCL between GPUs, gloo on CPUs) for
one rank per process, and LocalTransport for several slabs held by one process (the exchange
is then a device copy between the slabs' buffers).
"""
from dataclasses import dataclass

import torch

from . import _lib as L


@dataclass(frozen=True)
class Slab:
    k0: int          # first owned plane of the block
    k1: int          # one past the last owned plane
    ghost_lo: int    # ghost planes below (0 at the block's s = 0 face)
    ghost_hi: int    # ghost planes above (0 at the block's s = 1 face)

    @property
    def lo(self):
        """First plane of the block held locally."""
        return self.k0 - self.ghost_lo

    @property
    def hi(self):
        """One past the last plane of the block held locally."""
        return self.k1 + self.ghost_hi

    @property
    def planes(self):
        return self.hi - self.lo


def reach(order, operator="upwind"):
    """Ghost planes per inner slab end: the interior stencil's reach max(r, q)."""
    code = order + (L.SBP_TRADITIONAL if operator == "traditional" else 0)
    r = {2: 2, 3: 2, 4: 3, 5: 3, 6: 4, 7: 4, 102: 1, 104: 2, 106: 3}
    return r[code]


def metric_reach(order):
    """Planes of coordinates D_c of the metric operator reaches on each side: the metrics of
    every operator of a given order come from the upwind pair of that order."""
    return reach(order, "upwind")


def partition(ns, world, order, operator="upwind", min_face_planes=None):
    """Owned plane ranges of `world` slabs of a block of ns planes, as equal as the constraints
    allow: every slab owns at least `reach` planes (what it sends to a neighbour) and holds at
    least min_face_planes planes locally (default the operator's minimum grid size, which also
    covers the closure rows' taps of a slab at a face of the block)."""
    g = reach(order, operator)
    if min_face_planes is None:
        min_face_planes = sbp_min_nodes_py(order, operator)
    if world < 1:
        raise ValueError("world must be >= 1")
    if world == 1:
        return [Slab(0, ns, 0, 0)]
    base, extra = divmod(ns, world)
    sizes = [base + (1 if r < extra else 0) for r in range(world)]
    if min(sizes) < g:
        raise ValueError(f"{ns} planes over {world} slabs leaves fewer than {g} owned planes in one")
    out, k = [], 0
    for r, n in enumerate(sizes):
        out.append(Slab(k, k + n, 0 if r == 0 else g, 0 if r == world - 1 else g))
        k += n
    for sl in out:   # every slab's local grid has at least the operator's minimum size
        if sl.planes < min_face_planes:
            raise ValueError(f"a slab holds {sl.planes} planes, fewer than {min_face_planes}")
    return out


def sbp_min_nodes_py(order, operator="upwind"):
    code = order + (L.SBP_TRADITIONAL if operator == "traditional" else 0)
    return L.sbp_min_nodes(code)


def halo_ranges(sl, g):
    """Local plane ranges (start, stop) of the exchange: (send_down, recv_down, send_up, recv_up);
    None where the slab has no neighbour on that side."""
    P = sl.planes
    down = ((sl.ghost_lo, sl.ghost_lo + g), (0, g)) if sl.ghost_lo else (None, None)
    up = ((P - sl.ghost_hi - g, P - sl.ghost_hi), (P - g, P)) if sl.ghost_hi else (None, None)
    return down[0], down[1], up[0], up[1]


class DistTransport:
    """Halo exchange between ranks of torch.distributed (rank r holds slab r of the block)."""

    def __init__(self, dist, rank, world, group=None):
        self.dist, self.rank, self.world, self.group = dist, rank, world, group

    def exchange(self, view, sl, g):
        """view: the local state [nf][planes][nr][nq] (any device); fills its ghost planes."""
        sd, rd, su, ru = halo_ranges(sl, g)
        ops, recv = [], []
        if sd is not None:
            buf = view[:, sd[0]:sd[1]].contiguous()
            inb = torch.empty_like(buf)
            ops.append(self.dist.isend(buf, self.rank - 1, group=self.group))
            ops.append(self.dist.irecv(inb, self.rank - 1, group=self.group))
            recv.append((inb, rd))
        if su is not None:
            buf = view[:, su[0]:su[1]].contiguous()
            inb = torch.empty_like(buf)
            ops.append(self.dist.isend(buf, self.rank + 1, group=self.group))
            ops.append(self.dist.irecv(inb, self.rank + 1, group=self.group))
            recv.append((inb, ru))
        for op in ops:
            op.wait()
        for inb, (a, b) in recv:
            view[:, a:b].copy_(inb)


class LocalTransport:
    """Halo exchange among slabs held by one process: direct copies between their states."""

    @staticmethod
    def exchange_all(views, slabs, g):
        """views[r]: local state of slab r; fills every slab's ghost planes from its neighbours'
        owned planes (read before any ghost plane is written: owned and ghost planes differ)."""
        for r in range(len(slabs) - 1):
            sd_hi = halo_ranges(slabs[r], g)[2]        # slab r's last owned planes -> r+1's low ghosts
            rv_lo = halo_ranges(slabs[r + 1], g)[1]
            views[r + 1][:, rv_lo[0]:rv_lo[1]].copy_(views[r][:, sd_hi[0]:sd_hi[1]])
            sd_lo = halo_ranges(slabs[r + 1], g)[0]    # slab r+1's first owned planes -> r's high ghosts
            rv_hi = halo_ranges(slabs[r], g)[3]
            views[r][:, rv_hi[0]:rv_hi[1]].copy_(views[r + 1][:, sd_lo[0]:sd_lo[1]])


class SlabSolver:
    """One slab of a block on one device: an ElasticSolver over the slab's planes (owned and
    ghost) set up with sbp_set_slab.

    nodes: the block's (nq, nr, ns); slab: its Slab; coords, rlm: callables (k0, k1) -> (3, k1-k0,
    nr, nq) FP64 arrays of the block's node coordinates and (rho, lambda, mu) at planes k0..k1-1,
    so that no device holds the whole block.
    """

    def __init__(self, nodes, order, precision, bc, slab, coords, rlm, device="cuda", operator="upwind"):
        from .solver import ElasticSolver, _stream
        nq, nr, ns = nodes
        self.nodes, self.slab, self.order, self.operator = tuple(nodes), slab, order, operator
        self.g = reach(order, operator)
        self.s = ElasticSolver((nq, nr, slab.planes), order, precision, bc, device=device, operator=operator,
                               slab=(ns, slab.lo, slab.ghost_lo, slab.ghost_hi))
        # metrics at every local plane, ghost planes included: sbp_metrics on a window slab whose
        # owned planes cover this slab's local planes, with as many more planes of coordinates on
        # each inner side as D_c of the metric operator reaches (the rows of D_c are the block's;
        # the central operators' metric operator is the upwind pair of their order, which reaches
        # one plane further than they do)
        gm = max(self.g, metric_reach(order))
        w0, w1 = max(0, slab.lo - gm), min(ns, slab.hi + gm)
        glo, ghi = (slab.lo - w0 if w0 > 0 else 0), (w1 - slab.hi if w1 < ns else 0)
        win = ElasticSolver((nq, nr, w1 - w0), order, 64, bc, device=device, operator=operator,
                            slab=(ns, w0, glo, ghi) if (glo or ghi) else None)
        xyz = win.to_layout(torch.as_tensor(coords(w0, w1)), torch.float64)
        jwin = win.new_fields(10, torch.float64)
        L.sbp_metrics(win.h, xyz, jwin, _stream())
        if L.sbp_status(win.h, _stream()) & 2:
            raise L.SbpError(6, "non-positive Jacobian")
        jmet = self.s.new_fields(10, torch.float64)
        self.s.view(jmet, 10).copy_(win.view(jwin, 10)[:, slab.lo - w0:slab.lo - w0 + slab.planes])
        del win, xyz, jwin
        rlm_b = self.s.to_layout(torch.as_tensor(rlm(slab.lo, slab.hi)), torch.float64)
        L.sbp_set_material(self.s.h, jmet, rlm_b, _stream())
        if L.sbp_status(self.s.h, _stream()) & 6:
            raise L.SbpError(6, "invalid material")
        self.jmet = jmet

    def state(self):
        """The local state [9][planes][nr][nq] (owned and ghost planes)."""
        return self.s.state()

    def owned(self):
        """The owned planes of the state, [9][k1-k0][nr][nq]."""
        sl = self.slab
        return self.s.state()[:, sl.ghost_lo:sl.ghost_lo + (sl.k1 - sl.k0)]

    def stage(self, k, dt):
        self.s.rk_stage(k, dt)

    def energy(self):
        """This slab's part of the block's discrete energy (its owned planes)."""
        return self.s.energy()


def step_local(solvers, n, dt):
    """n Runge-Kutta steps of slabs held by one process (LocalTransport): every stage on every
    slab, then the halo exchange of the new states."""
    g = solvers[0].g
    slabs = [s.slab for s in solvers]
    for _ in range(n):
        for k in range(5):
            for s in solvers:
                s.stage(k, dt)
            LocalTransport.exchange_all([s.state() for s in solvers], slabs, g)


def step_dist(solver, transport, n, dt):
    """n Runge-Kutta steps of this rank's slab: every stage, then the halo exchange."""
    for _ in range(n):
        for k in range(5):
            solver.stage(k, dt)
            transport.exchange(solver.state(), solver.slab, solver.g)
