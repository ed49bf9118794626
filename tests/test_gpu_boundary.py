"""The C ABI's host-facing calls on the GPU: state upload and download with host or device
buffers (sbp_set_state / sbp_get_state), receivers placed by physical position
(sbp_set_receivers_xyz) and traces copied out by sbp_record_receivers.

The receivers are the paper's stations (Section 7: particle velocity at surface nodes).  The
nearest node is checked against a brute-force search over the same face in numpy; the traces of
a short FP64 run against the oracle's traces at the same nodes (1e-11, as for the other runs)."""
import numpy as np
import pytest
import torch

from oracle.solver import OracleSolver
from workloads.fields import gaussian_pulse, random_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium
from workloads.timestep import stable_dt

pytestmark = pytest.mark.gpu

BC = [("char", 0.0)] * 5 + [("free",)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _setup(nodes, order, prec, ext=(1000.0, 1100.0, 900.0), batch=1):
    from paper_2011_02600_gb300 import ElasticSolver
    X = node_coordinates(make_map("curvy", ext), nodes)
    mat = make_medium("smooth_gradient", Lz=ext[2])(*X)
    s = ElasticSolver(nodes, order, prec, BC, batch=batch)
    s.setup(torch.from_numpy(np.stack(X)), torch.from_numpy(np.stack(mat)))
    return s, X, mat


@pytest.mark.parametrize("prec", [32, 64])
def test_state_upload_download_round_trip(prec):
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    nodes = (37, 19, 14)
    s, X, mat = _setup(nodes, 4, prec, batch=2)
    npdt = np.float32 if prec == 32 else np.float64
    Q = np.concatenate([random_state(nodes, 5), random_state(nodes, 6)]).astype(npdt)   # [18][ns][nr][nq]
    # host, packed
    s.upload_state(Q)
    assert np.array_equal(s.state(0).cpu().numpy(), Q[:9]) and np.array_equal(s.state(1).cpu().numpy(), Q[9:])
    back = s.download_state(np.zeros_like(Q))
    assert np.array_equal(back, Q)
    # device, packed
    dev = torch.from_numpy(Q).cuda()
    s.upload_state(dev * 2)
    out = s.download_state(torch.zeros_like(dev))
    assert torch.equal(out, dev * 2)
    # host, grid layout (pinned), and a step after the upload equals a step after a torch copy
    flat = torch.zeros(18 * s.fs, dtype=s.dtype).pin_memory()
    s.view(flat, 18).copy_(torch.from_numpy(Q))
    L.sbp_set_state(s.h, flat, L.SBP_MEM_HOST, _stream())
    s.step(2, 1e-4)
    got = torch.zeros(18 * s.fs, dtype=s.dtype).pin_memory()
    L.sbp_get_state(s.h, got, L.SBP_MEM_HOST, _stream())
    # the same download enqueued without waiting (SBP_MEM_ASYNC), read after a synchronisation
    got_async = torch.zeros(18 * s.fs, dtype=s.dtype).pin_memory()
    L.sbp_get_state(s.h, got_async, L.SBP_MEM_HOST | L.SBP_MEM_ASYNC, _stream())
    torch.cuda.synchronize()
    assert torch.equal(got_async, got)
    s2, _, _ = _setup(nodes, 4, prec, batch=2)
    s2.qbuf[0].copy_(flat.cuda())
    s2.step(2, 1e-4)
    assert torch.equal(s2.view(s2.qbuf[s2.current], 18).cpu(), s.view(got, 18))


def test_copy_calls_reject_bad_arguments():
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    s, X, mat = _setup((20, 20, 20), 4, 32)
    buf = np.zeros(9 * 20 ** 3, dtype=np.float32)
    for fn, args, code in [(L.sbp_set_state, (None, 3, _stream()), 1),
                           (L.sbp_set_state, (buf, 8, _stream()), 1),
                           (L.sbp_set_state, (buf, L.SBP_MEM_ASYNC, _stream()), 1),
                           (L.sbp_get_state, (buf, 8, _stream()), 1),
                           (L.sbp_record_receivers, (buf, 1, _stream()), 5)]:
        with pytest.raises(L.SbpError) as e:
            fn(s.h, *args)
        assert e.value.code == code
    coords = s.to_layout(torch.from_numpy(np.stack(X)), torch.float64)
    for pts, face in [([[0.0, 0.0, np.nan]], 5), ([[0.0, 0.0, 0.0]], 6), ([[0.0, 0.0, 0.0]], -2)]:
        with pytest.raises(L.SbpError) as e:
            L.sbp_set_receivers_xyz(s.h, pts, coords, face, None, 10)
        assert e.value.code == 1


@pytest.mark.parametrize("face", [5, 0, -1])
def test_receivers_by_position_pick_the_nearest_node(face):
    nodes = (33, 29, 25)
    s, X, mat = _setup(nodes, 6, 32)
    x, y, z = (np.asarray(c) for c in X)
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(x.min(), x.max(), 40), rng.uniform(y.min(), y.max(), 40),
                    rng.uniform(z.min(), z.max(), 40)], axis=1)
    ijk = s.set_receivers_at(pts, np.stack(X), 5, face=face)
    nq, nr, ns = nodes
    K, Jj, I = np.meshgrid(np.arange(ns), np.arange(nr), np.arange(nq), indexing="ij")
    sel = np.ones_like(I, dtype=bool)
    if face >= 0:
        idx = (I, I, Jj, Jj, K, K)[face]
        sel = idx == (0 if face % 2 == 0 else nodes[face // 2] - 1)
    cand = np.flatnonzero(sel.ravel())                        # ascending [s][r][q] order
    P = np.stack([x.ravel()[cand], y.ravel()[cand], z.ravel()[cand]], axis=1)
    for r, p in enumerate(pts):
        d2 = ((P - p) ** 2).sum(axis=1)
        t = cand[np.flatnonzero(d2 == d2.min())[0]]
        want = (t % nq, (t // nq) % nr, t // (nq * nr))
        assert tuple(ijk[r]) == want, (r, tuple(ijk[r]), want)


def test_recorded_traces_match_the_oracle():
    """Receivers placed by position on the free surface, FP64 run of a pulse for 25 steps: the
    traces copied out (host and device) equal the oracle's traces at the chosen nodes."""
    nodes, order = (29, 27, 25), 4
    ext = (2000.0, 2000.0, 1500.0)
    s, X, mat = _setup(nodes, order, 64, ext=ext)
    dt = stable_dt(*X, *mat, 0.5)
    Q0 = np.stack(gaussian_pulse(*X, (1000.0, 1000.0, -500.0), 150.0))
    s.upload_state(Q0)
    pts = [[500.0, 700.0, 0.0], [1500.0, 1000.0, 50.0], [1000.0, 1000.0, 0.0]]
    ijk = s.set_receivers_at(pts, np.stack(X), 25, face=5)
    assert all(k == nodes[2] - 1 for _, _, k in ijk)
    s.step(25, dt)
    host = s.record_receivers(host=True)
    dev = s.record_receivers(host=False)
    assert np.array_equal(host, dev.cpu().numpy())
    orc = OracleSolver(order, *X, mat, BC)
    orc.Q[:] = Q0
    orc.receivers = [tuple(int(v) for v in r) for r in ijk]
    orc.step(dt, 25)
    want = np.stack(orc.traces, axis=-1)
    assert np.abs(host - want).max() / np.abs(want).max() < 1e-11
