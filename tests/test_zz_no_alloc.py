"""The allocation-free energy entry point (sbp_energy_noalloc) against sbp_energy.

Some callers cannot let a library call cudaMalloc: frameworks that own a pooled
allocator, or code that works within device memory reserved up front.  For them
sbp_energy_noalloc computes the discrete energy with a static device scratch
array instead of the buffer sbp_energy allocates when a grid is bound.  This
file is collected last so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest
import torch

from workloads.fields import random_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_02600_gb300 import _lib as L
    return L


@pytest.mark.parametrize("prec,order,nodes", [(64, 4, (37, 19, 14)), (32, 6, (41, 29, 23))])
def test_noalloc_energy_matches_allocating_entry_point(lib, prec, order, nodes):
    from paper_2011_02600_gb300 import ElasticSolver
    from paper_2011_02600_gb300.solver import _stream
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    s = ElasticSolver(nodes, order, prec, [("char", 0.0)] * 5 + [("free",)])
    s.setup(torch.from_numpy(np.stack(X)), torch.from_numpy(np.stack(mat)))
    s.set_state(torch.from_numpy(random_state(nodes, 21, 1.0, 1.0e6)))
    want = s.energy()
    q = s.qbuf[s.current]
    got = [lib.sbp_energy_noalloc(q, s.mat, nodes, s.ldq, s.fs, order, prec, 0, _stream()) for _ in range(2)]
    for g in got:
        assert abs(g - want) <= 1e-12 * abs(want), (g, want)
    # a different partial-sum count still gives the energy to rounding
    g3 = lib.sbp_energy_noalloc(q, s.mat, nodes, s.ldq, s.fs, order, prec, 4096, _stream())
    assert abs(g3 - want) <= 1e-12 * abs(want)


def test_noalloc_energy_rejects_sizes_beyond_its_scratch(lib):
    from paper_2011_02600_gb300 import ElasticSolver
    from paper_2011_02600_gb300.solver import _stream
    nodes = (16, 16, 16)
    s = ElasticSolver(nodes, 6, 32)
    with pytest.raises(lib.SbpError) as e:
        lib.sbp_energy_noalloc(s.qbuf[0], s.mat, nodes, s.ldq, s.fs, 6, 32, 4097, _stream())
    assert e.value.code == 1 and "4096" in str(e.value)
    with pytest.raises(lib.SbpError) as e:
        lib.sbp_energy_noalloc(s.qbuf[0], s.mat, nodes, s.ldq, 1 << 31, 6, 32, 0, _stream())
    assert e.value.code == 1
