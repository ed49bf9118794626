"""Failure detection on the device, without a GPU fault.

Every device-side finding is a bit in the grid's status word, read by sbp_status:
a non-finite state (energy reduction), a non-positive Jacobian (metrics), invalid
moduli (material), and a tile copy that never lands (the tiled kernel's bounded
mbarrier wait).  The last is exercised by sbp_selftest_wait_timeout, a bounded wait on
a barrier that nothing completes; afterwards the context must still compute.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _grid(nodes=(20, 18, 17), order=4, precision=32, X=None, mat=None):
    from paper_2011_02600_gb300 import ElasticSolver
    from workloads.fields import random_state
    nq, nr, ns = nodes
    if X is None:
        z, y, x = np.meshgrid(np.linspace(-1000, 0, ns), np.linspace(0, 1200, nr), np.linspace(0, 1300, nq),
                              indexing="ij")
        X = np.stack([x, y, z])
    if mat is None:
        mat = np.stack([np.full((ns, nr, nq), 2700.0), np.full((ns, nr, nq), 3.24e10),
                        np.full((ns, nr, nq), 3.24e10)])
    s = ElasticSolver(nodes, order, precision, [("char", 0.0)] * 5 + [("free",)])
    s.setup(torch.from_numpy(X), torch.from_numpy(mat))
    s.set_state(torch.from_numpy(random_state(nodes, 3, 1.0, 1.0e6)))
    return s


def test_wait_timeout_is_reported_and_the_context_survives():
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    s = _grid()
    q = torch.from_numpy(np.random.default_rng(1).normal(size=(9,) + (17, 18, 20)))
    r0 = s.rhs(q).clone()
    assert s.status() == 0
    L.sbp_selftest_wait_timeout(s.h, 2000, _stream())
    assert s.status() == 8           # SBP_STATUS_TIMEOUT, and only that
    assert s.status() == 0           # reading clears it
    r1 = s.rhs(q)
    assert torch.equal(r0, r1)
    with pytest.raises(L.SbpError):
        L.sbp_selftest_wait_timeout(s.h, 0, _stream())


def test_nonfinite_state_is_reported():
    from paper_2011_02600_gb300 import _lib as L
    s = _grid()
    st = s.state()
    st[4, 3, 5, 7] = float("nan")
    with pytest.raises(L.SbpError) as ex:
        s.energy()
    assert ex.value.code == 4        # SBP_ERR_NONFINITE
    assert s.status() & 1            # SBP_STATUS_NONFINITE


def test_folded_mesh_is_reported():
    from paper_2011_02600_gb300 import _lib as L
    nodes = (20, 18, 17)
    nq, nr, ns = nodes
    z, y, x = np.meshgrid(np.linspace(-1000, 0, ns), np.linspace(0, 1200, nr), np.linspace(0, 1300, nq),
                          indexing="ij")
    x = x.copy()
    x[:, :, 10:] = x[:, :, 10:][:, :, ::-1] - 700.0      # the q lines fold back: J < 0 there
    with pytest.raises(L.SbpError) as ex:
        _grid(nodes, X=np.stack([x, y, z]))
    assert ex.value.code == 6


def test_invalid_material_is_reported():
    from paper_2011_02600_gb300 import _lib as L
    nodes = (20, 18, 17)
    nq, nr, ns = nodes
    mat = np.stack([np.full((ns, nr, nq), 2700.0), np.full((ns, nr, nq), 3.24e10), np.full((ns, nr, nq), 3.24e10)])
    mat[2, 8, 9, 10] = -1.0e9                              # negative shear modulus at one node
    with pytest.raises(L.SbpError) as ex:
        _grid(nodes, mat=mat)
    assert ex.value.code == 6


def test_checkpoint_resume_is_bit_identical_fp64(tmp_path):
    """save_state between steps and load_state into a fresh grid continue the run bit for bit
    (FP64), time and step counter included; a grid of another shape is refused."""
    from paper_2011_02600_gb300.checkpoint import CheckpointError
    a = _grid(precision=64)
    b = _grid(precision=64)
    dt = 1e-4
    a.step(12, dt)
    b.step(5, dt)
    path = str(tmp_path / "run.ckpt")
    b.save_state(path)
    c = _grid(precision=64)
    c.set_state(torch.zeros_like(c.state()))
    c.load_state(path)
    c.step(7, dt)
    assert torch.equal(a.state(), c.state())
    assert torch.equal(a.view(a.dq, 9), c.view(c.dq, 9))
    from paper_2011_02600_gb300 import _lib as L
    assert L.sbp_get_time(a.h) == L.sbp_get_time(c.h)
    other = _grid(nodes=(21, 18, 17), precision=64)
    with pytest.raises(CheckpointError):
        other.load_state(path)


def test_periodic_check_stops_a_nonfinite_run():
    from paper_2011_02600_gb300 import _lib as L
    s = _grid()
    s.step(3, 1e-4, check_every=2)           # finite: passes
    s.state()[2, 4, 5, 6] = float("inf")
    with pytest.raises(L.SbpError) as ex:
        s.step(10, 1e-4, check_every=4)
    assert ex.value.code == 4
