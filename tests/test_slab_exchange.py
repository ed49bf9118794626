"""The s-slab decomposition and its halo exchange (slab.py) on CPU ranks (gloo, world sizes 2
and 4), against the undivided block.

Every rank holds its slab's planes plus `reach` ghost planes at each inner end, advances its
owned planes by the oracle's Runge-Kutta stages (evaluated on the block with the rank's planes
in place: every tap of an owned plane lies inside the slab) and, after every stage, exchanges
its first and last `reach` owned planes with its neighbours through torch.distributed.  After
three steps the owned planes gathered from all ranks equal the single-domain oracle run bit
for bit (FP64), for upwind orders 4 and 6 and a traditional operator.  The partition's and the
exchange ranges' rules are checked directly as well."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {"o4": (4, "upwind", (11, 12, 40)), "o6": (6, "upwind", (16, 16, 70)), "t4": (4, "traditional", (12, 11, 44))}
BC = [("char", 0.0), ("char", 0.2), ("char", -0.3), ("char", 0.0), ("char", 0.0), ("free",)]
STEPS, DT = 3, 2.0e-4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(case):
    sys.path.insert(0, ROOT)
    from oracle.elastic import Scheme
    from oracle.metrics import metrics
    from workloads.fields import random_state
    from workloads.geometry import make_map, node_coordinates
    from workloads.media import make_medium
    order, op, nodes = CASES[case]
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    J, a = metrics(*X, order)
    return order, op, nodes, Scheme(order, nodes, op), J, a, mat, random_state(nodes, 41, 1.0, 1.0e6)


def _oracle_run(case):
    from oracle import rk
    from oracle.elastic import rhs
    order, op, nodes, sch, J, a, mat, Q = _problem(case)
    Q, dQ = Q.copy(), np.zeros_like(Q)
    for _ in range(STEPS):
        rk.rk_step(Q, dQ, 0.0, DT, lambda q, t: rhs(q, sch, J, a, mat, BC))
    return Q


def _rank(rank, world, port, case, out):
    try:
        _rank_body(rank, world, port, case, out)
    except BaseException as e:   # report instead of leaving rank 0 waiting
        out.put(f"rank {rank}: {type(e).__name__}: {e}")
        raise


def _rank_body(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import rk
    from oracle.elastic import rhs
    from paper_2011_02600_gb300 import slab as S
    order, op, nodes, sch, J, a, mat, Q0 = _problem(case)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    slabs = S.partition(nodes[2], world, order, op)
    sl, g = slabs[rank], S.reach(order, op)
    # the rank's local arrays: its planes of the block, the ghost planes included
    q = torch.from_numpy(Q0[:, sl.lo:sl.hi].copy())
    dq = torch.zeros_like(q)
    own = slice(sl.ghost_lo, sl.ghost_lo + sl.k1 - sl.k0)
    tr = S.DistTransport(dist, rank, world)
    for _ in range(STEPS):
        for k in range(5):
            # the oracle's right-hand side with this rank's planes in place in the block
            emb = np.zeros_like(Q0)
            emb[:, sl.lo:sl.hi] = q.numpy()
            d = rhs(emb, sch, J, a, mat, BC)[:, sl.lo:sl.hi]
            dq[:, own] = torch.from_numpy(rk.A[k] * dq[:, own].numpy() + DT * d[:, own])
            q[:, own] += rk.B[k] * dq[:, own]
            tr.exchange(q, sl, g)
    mine = q[:, own].contiguous()
    if rank == 0:   # collect the owned planes (slabs may differ in size by one plane)
        parts = [mine]
        for r in range(1, world):
            buf = torch.zeros(9, slabs[r].k1 - slabs[r].k0, nodes[1], nodes[0], dtype=torch.float64)
            dist.recv(buf, r)
            parts.append(buf)
        out.put(torch.cat(parts, dim=1).numpy())
    else:
        dist.send(mine, 0)
    dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("world", [2, 4])
def test_slab_run_matches_undivided_oracle(case, world):
    torch = pytest.importorskip("torch")
    from paper_2011_02600_gb300 import build as B
    B.build()
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
    assert not isinstance(got, str), got
    assert all(p.exitcode == 0 for p in procs)
    want = _oracle_run(case)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_partition_rules():
    from paper_2011_02600_gb300 import build as B
    B.build()
    from paper_2011_02600_gb300 import slab as S
    for ns, world, order in [(401, 2, 6), (401, 8, 6), (97, 4, 4), (40, 3, 2), (70, 4, 6)]:
        sl = S.partition(ns, world, order)
        g = S.reach(order)
        assert sl[0].k0 == 0 and sl[-1].k1 == ns
        assert all(a.k1 == b.k0 for a, b in zip(sl, sl[1:]))
        assert sl[0].ghost_lo == 0 and sl[-1].ghost_hi == 0
        assert all(s.ghost_lo == g for s in sl[1:]) and all(s.ghost_hi == g for s in sl[:-1])
        sizes = [s.k1 - s.k0 for s in sl]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= g
    with pytest.raises(ValueError):
        S.partition(20, 8, 6)          # fewer than 4 owned planes per slab
    with pytest.raises(ValueError):
        S.partition(32, 4, 6)          # a face slab would hold 8 + 4 < 16 planes


def test_halo_ranges_pair_up():
    """What a slab sends down is what its lower neighbour receives as its upper ghosts (same
    planes of the block), and the same upwards; the sent planes are owned, the received ones
    are the ghost planes."""
    from paper_2011_02600_gb300 import build as B
    B.build()
    from paper_2011_02600_gb300 import slab as S
    for ns, world, order in [(70, 4, 6), (97, 3, 4), (401, 8, 6)]:
        sl, g = S.partition(ns, world, order), S.reach(order)
        for r in range(world - 1):
            lo, hi = sl[r], sl[r + 1]
            su, ru = S.halo_ranges(lo, g)[2], S.halo_ranges(lo, g)[3]
            sd, rd = S.halo_ranges(hi, g)[0], S.halo_ranges(hi, g)[1]
            assert [lo.lo + k for k in range(*su)] == [hi.lo + k for k in range(*rd)]
            assert [hi.lo + k for k in range(*sd)] == [lo.lo + k for k in range(*ru)]
            assert all(lo.k0 <= lo.lo + k < lo.k1 for k in range(*su))
            assert all(not (hi.k0 <= hi.lo + k < hi.k1) for k in range(*rd))
