"""The s-slab decomposition on the GPU: slabs of one block held by one process (the exchange is
a device copy between the slabs' states, slab.LocalTransport), each with the stage kernel
computing its owned planes only (sbp_set_slab).  After several Runge-Kutta steps every slab's
owned planes equal the undivided block's bit for bit (FP64 and FP32: the same arithmetic per
node), and the slabs' energies add up to the block's (1e-13, different summation order).  No
kernel waits on another slab's kernels: the slabs' stages and copies run one after another."""
import numpy as np
import pytest
import torch

from workloads.fields import random_state, smooth_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium

pytestmark = pytest.mark.gpu

BC = [("char", 0.0), ("char", 0.2), ("char", -0.3), ("char", 0.0), ("char", 0.0), ("free",)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("order,operator,nodes,world", [(6, "upwind", (41, 29, 70), 3), (4, "upwind", (37, 19, 60), 4),
                                                        (6, "traditional", (33, 20, 50), 2)])
@pytest.mark.parametrize("prec", [64, 32])
def test_slabs_match_the_undivided_block(order, operator, nodes, world, prec):
    from paper_2011_02600_gb300 import ElasticSolver
    from paper_2011_02600_gb300 import slab as S
    X = np.stack(node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes))
    mat = np.stack(make_medium("smooth_gradient", Lz=900.0)(*X))
    K, Jj, I = np.meshgrid(np.arange(nodes[2]), np.arange(nodes[1]), np.arange(nodes[0]), indexing="ij")
    Q0 = random_state(nodes, 5, 1.0, 1.0e6) if prec == 64 else np.stack(smooth_state(nodes, 5, I, Jj, K))
    whole = ElasticSolver(nodes, order, prec, BC, operator=operator)
    whole.setup(torch.from_numpy(X), torch.from_numpy(mat))
    whole.set_state(torch.from_numpy(Q0))
    slabs = S.partition(nodes[2], world, order, operator)
    sol = [S.SlabSolver(nodes, order, prec, BC, sl, lambda a, b: X[:, a:b], lambda a, b: mat[:, a:b],
                        operator=operator) for sl in slabs]
    for s in sol:
        s.state().copy_(torch.from_numpy(Q0[:, s.slab.lo:s.slab.hi]))
    dt = 2.0e-4
    e_whole = whole.energy()
    e_slabs = sum(s.energy() for s in sol)
    assert abs(e_slabs - e_whole) < 1e-13 * e_whole
    whole.step(4, dt)
    S.step_local(sol, 4, dt)
    ref = whole.state()
    for s in sol:
        sl = s.slab
        assert torch.equal(s.owned(), ref[:, sl.k0:sl.k1]), sl
    e_whole = whole.energy()
    e_slabs = sum(s.energy() for s in sol)
    assert abs(e_slabs - e_whole) < 1e-12 * e_whole


def test_slab_refusals():
    """What the slab grids do not run says so (UNSUPPORTED), and bad slab shapes are refused."""
    from paper_2011_02600_gb300 import ElasticSolver
    from paper_2011_02600_gb300 import _lib as L
    nodes = (20, 20, 24)
    s = ElasticSolver(nodes, 4, 64, BC, slab=(60, 10, 3, 3))
    src = dict(ref=(0.5, 0.5, 0.5), moment=[1.0] * 6, stf=0, f0=1.0, t0=1.0)
    for fn, args in [(L.sbp_set_sources, ([src], s.new_fields(10, torch.float64), 0)),
                     (L.sbp_rhs_adjoint, (s.new_fields(9), s.new_fields(9), s.new_fields(9), 0))]:
        with pytest.raises(L.SbpError) as e:
            fn(s.h, *args)
        assert e.value.code == 2
    # the central operator of order 6 reaches 3 planes, its metric operator (the upwind pair of
    # order 6) 4: metrics on a slab with 3 ghost planes would read past the local planes
    t = ElasticSolver(nodes, 6, 64, BC, slab=(60, 10, 3, 3), operator="traditional")
    with pytest.raises(L.SbpError) as e:
        L.sbp_metrics(t.h, t.new_fields(3, torch.float64), t.new_fields(10, torch.float64), 0)
    assert e.value.code == 1
    h = L.sbp_create_grid(nodes, 4, 64, BC)
    for bad in [(60, 10, 2, 3), (60, 0, 3, 3), (60, 40, 3, 0), (60, 50, 3, 3), (8, 0, 0, 3)]:
        with pytest.raises(L.SbpError) as e:
            L.sbp_set_slab(h, *bad)
        assert e.value.code == 1, bad
    L.sbp_destroy(h)
