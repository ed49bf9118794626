"""The receiver misfit on the GPU: the sum over receivers and components of 1/2 w (v - d)^2, with
its adjoint source w (v - d) at each receiver node.  The paper has no adjoint; the misfit is the
plain definition used by the gradient.  Checked here:

* receivers that share a node each add their own adjoint source there;
* a rejected receiver list leaves the current receivers in place.

The expected values are formed here from the state read back and the data (no oracle needed:
the misfit is a plain sum at the receiver nodes).
"""
import numpy as np
import pytest
import torch

from workloads.fields import random_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium

pytestmark = pytest.mark.gpu

NODES, ORDER = (16, 17, 16), 4
# three receivers on the node (3, 4, 15), one elsewhere
REC = [(3, 4, 15), (9, 2, 15), (3, 4, 15), (3, 4, 15)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _case(prec):
    from paper_2011_02600_gb300 import ElasticSolver
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), NODES)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    s = ElasticSolver(NODES, ORDER, prec, [("free",)] * 6)
    s.setup(torch.from_numpy(np.stack(X)), torch.from_numpy(np.stack(mat)))
    q = s.to_layout(torch.from_numpy(random_state(NODES, 7, 1.0, 1.0e6)), s.dtype)
    s.set_receivers(REC, 1)
    data = torch.from_numpy(np.random.default_rng(5).normal(size=(len(REC), 3))).to(s.device)
    return s, q, data


def _expected(qv, d, w):
    ub = np.zeros_like(qv)
    acc = np.zeros(len(REC) * 3)
    for r, (i, j, k) in enumerate(REC):
        for c in range(3):
            diff = qv[c, k, j, i] - d[r, c]
            ub[c, k, j, i] += w * diff
            acc[3 * r + c] = 0.5 * w * diff * diff
    return ub, acc


@pytest.mark.parametrize("prec", [64, 32])
def test_receivers_on_one_node_add_their_adjoint_sources(prec):
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    s, q, data = _case(prec)
    acc = torch.zeros(len(REC) * 3, dtype=torch.float64, device=s.device)
    ubar = s.new_fields(9)
    w = 0.25
    L.sbp_misfit(s.h, q, data.reshape(-1), w, acc, ubar, _stream())
    torch.cuda.synchronize()
    qv = s.view(q, 9).double().cpu().numpy()
    ub_want, acc_want = _expected(qv, data.cpu().numpy(), w)
    ub = s.view(ubar, 9).double().cpu().numpy()
    tol = 1e-14 if prec == 64 else 1e-6
    assert np.abs(ub - ub_want).max() <= tol * np.abs(ub_want).max()
    # every node but the two receiver nodes is untouched
    assert np.count_nonzero(ub) == np.count_nonzero(ub_want) == 6
    assert np.allclose(acc.cpu().numpy(), acc_want, rtol=1e-12, atol=0.0)


def test_rejected_receiver_list_keeps_the_current_receivers():
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    s, q, data = _case(64)
    with pytest.raises(L.SbpError):
        L.sbp_set_receivers(s.h, [(NODES[0], 0, 0)], s.traces, 1)
    acc = torch.zeros(len(REC) * 3, dtype=torch.float64, device=s.device)
    L.sbp_misfit(s.h, q, data.reshape(-1), 1.0, acc, None, _stream())
    torch.cuda.synchronize()
    _, acc_want = _expected(s.view(q, 9).double().cpu().numpy(), data.cpu().numpy(), 1.0)
    assert np.allclose(acc.cpu().numpy(), acc_want, rtol=1e-12, atol=0.0)


def test_zero_steps_and_a_zero_state():
    """Degenerate calls: zero steps leave state, time and step counter as they are; the zero
    state is a fixed point of the scheme without a source (L is linear)."""
    from paper_2011_02600_gb300 import _lib as L
    s, _, _ = _case(64)
    Q = random_state(NODES, 8, 1.0, 1.0e6)
    s.set_state(torch.from_numpy(Q))
    s.set_time(0.5, 3)
    s.step(0, 1.0e-4)
    torch.cuda.synchronize()
    assert np.array_equal(s.state().cpu().numpy(), Q)
    assert L.sbp_get_time(s.h) == (0.5, 3)
    s.set_state(torch.zeros((9,) + Q.shape[1:], dtype=torch.float64))
    s.step(2, 1.0e-4)
    torch.cuda.synchronize()
    assert not s.state().cpu().numpy().any()
    assert L.sbp_get_time(s.h)[1] == 5
