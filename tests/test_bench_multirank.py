"""The multi-process paths of bench.py on CPU (gloo, world size 2): the slowest rank's time
is every rank's (a rank without one counts as infinitely slow), the end-to-end record is the
whole job's, the ranks of a node split its free host memory for pinned buffers, and the
reference arm prints one line from rank 0 while the other ranks exit without work."""
import json
import math
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    got = bench.max_over_ranks(values[rank], dist)
    dist.destroy_process_group()
    out.put((rank, got))


def test_max_over_ranks_gloo_world2():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    values = [3.5, 7.25]
    procs = [mp.Process(target=_rank, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 7.25, 1: 7.25}


def test_max_over_ranks_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None) == 2.5


def test_reference_arm_under_torchrun_world2():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env={**os.environ, "OMP_NUM_THREADS": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Mnode-stage/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_max_over_ranks_counts_a_rank_without_a_time_as_slowest():
    """A rank whose end-to-end leg failed reports inf; the job then has no pipelined time."""
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    values = [12.5, math.inf]
    procs = [mp.Process(target=_rank, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: math.inf, 1: math.inf}


def test_e2e_record_whole_job():
    """The e2e figure is the job's: world x nodes x 5 stages per step over the slowest rank's
    time per step, and world x the state's bytes each way."""
    sys.path.insert(0, ROOT)
    import bench
    nodes, nbytes = 1000, 36000
    one = bench.e2e_record(nodes, 1, nbytes, 4.0, 2.0, 3, 3, 9)
    assert one["value"] == pytest.approx(nodes * 5 / 2e-3 / 1e6)
    assert one["h2d_bytes_per_step"] == one["d2h_bytes_per_step"] == nbytes
    assert one["grids"] == 3 and one["steps"] == 9
    assert one["sequential_one_grid"]["value"] == pytest.approx(nodes * 5 / 4e-3 / 1e6)
    four = bench.e2e_record(nodes, 4, nbytes, 4.0, 2.0, 2, 3, 6)
    assert four["value"] == pytest.approx(4 * one["value"])
    assert four["h2d_bytes_per_step"] == 4 * nbytes and "each of the 4 ranks" in four["what"]
    # no pipelined time on some rank: the sequential figure, with the reason
    seq = bench.e2e_record(nodes, 2, nbytes, 4.0, math.inf, 1, 3, 0, note="no room for a second grid")
    assert seq["value"] == pytest.approx(2 * nodes * 5 / 4e-3 / 1e6)
    assert "grids" not in seq and seq["note"] == "no room for a second grid"
    # no time at all: no value, the reason kept
    none = bench.e2e_record(nodes, 1, nbytes, math.inf, math.inf, 1, 3, 0, note="pinning failed")
    assert none["value"] is None and none["error"] == "pinning failed"
    assert json.loads(json.dumps(one)) == one


def test_host_memory_share_splits_among_the_node_ranks():
    sys.path.insert(0, ROOT)
    import bench
    whole = bench.host_memory_share(1)
    assert whole > 0
    if math.isfinite(whole):
        assert bench.host_memory_share(4) == pytest.approx(whole / 4, rel=0.05)
    assert bench.host_memory_share(0) > 0
