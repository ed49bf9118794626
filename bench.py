"""Throughput of the fused RHS + Runge-Kutta stage on one GB300.

Workload: 1025 x 1025 x 401 nodes (421M), order-6 upwind SBP, FP32, 60 x 60 x 24 km
block with a seeded sum-of-sinusoids top surface (free) and absorbing faces
elsewhere, von Karman perturbed gradient medium.  A step is one full
Runge-Kutta step: five fused stages over every node (one launch of the tiled
stage kernel per stage; the grid is a topography map, so the stage reads the 4
metric fields of that path and its roofline counts 172 B per node-stage, 136 in
the first stage).  Metric: million node-stage updates per second,
nodes * 5 * steps / time.  The end-to-end figure moves every step's state in from
and out to pinned host memory through the C ABI, with two or three grids taking
the steps in turn so that copies and steps overlap.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload adjoint129_o4 [--adj-steps N]
    python bench.py --workload surrogate97_o4

The second form times one misfit gradient of the adjoint workload (129 x 129 x 97, order 4,
FP32 forward with FP64 misfit, 1500 steps, sqrt(N) checkpoints, its eight sources as one batch):
forward run, checkpoint recomputation and adjoint stages, with the adjoint stage kernels' roofline.  The third times the
surrogate network's training iterations at full size and its largest GEMM against the BF16 peak.

One JSON line on rank 0.  With --gpus N > 1 (torchrun) every rank runs an
independent replica of the workload on its own GPU ("replicas only": the
single-block path has no exchange step) and the value is the sum over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoint-updates/s per RK stage"
UNIT = "Mnode-stage/s"
WORKLOAD = "topo1025_o6_fp32"
BYTES_PER_NODE_STAGE = 192        # 48 FP32 values per node per stage (algorithmic)
BYTES_PER_NODE_STAGE0 = 156       # first stage: A_0 = 0, the RK register is not read
NOMINAL_HBM_GBS = 7900.0          # HBM3e nominal, for the second fraction
L2_BYTES = 129e6                  # L2 capacity: the bench inputs must exceed it (no flush between steps)
FLOP_PER_NODE_STAGE = 444         # order 6, interior node, counted from the tiled kernel's arithmetic (an FMA
                                  # is 2): fluxes F_q, F_r on the tile and halo (1.19 + 1.75 per node) and F_s,
                                  # 15 each: 59; D- and D+ on 3 axes x 3 components, 7 taps and a scaling: 270;
                                  # strain rows 54; P~ 16; Runge-Kutta update 45
# The topography-map path (x = L_x q, y = L_y r: a_q = (a_q,x, 0, 0), a_r = (0, c a_q,x, 0)) reads 4
# metric fields instead of 9: 43 values per node and stage, 34 in stage 0; its fluxes F_q, F_r take
# 3 and 4 flop and the q and r strain rows 6 and 7, so 388 flop per node and stage.
BYTES_PER_NODE_STAGE_TOPO = 172
BYTES_PER_NODE_STAGE0_TOPO = 136
FLOP_PER_NODE_STAGE_TOPO = 388
FP64_NOMINAL_TFLOPS = 1.25        # GB300 FP64 nominal; the roofline uses the rate measured on the device


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, dist, device="cpu"):
    """The largest x over all ranks (the job's time is the slowest rank's); x itself when
    there is no process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_memory_share(local_world):
    """Bytes of host memory this rank may pin: what the node has free now, split evenly among
    the ranks on the node (they all pin at once); unlimited when the platform does not say."""
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return math.inf
    return avail / max(1, local_world)


def e2e_record(nodes, world, nbytes, seq_ms, e_ms, grids, seq_steps, e_steps, note=None):
    """The bench line's `e2e` object from the job's milliseconds per step (the slowest rank's;
    inf where some rank has no number): the pipelined figure when every rank has one, else the
    one-grid sequential figure, else none.  Each of the `world` ranks streams its own grid's
    state of `nbytes` in and out every step, so the job moves world x nbytes each way."""
    def rate(ms):
        return world * nodes * 5 / (ms / 1e3) / 1e6
    ranks = f" on each of the {world} ranks" if world > 1 else ""
    if math.isfinite(e_ms) and math.isfinite(seq_ms):
        rec = {"value": rate(e_ms), "unit": UNIT, "h2d_bytes_per_step": world * nbytes,
               "d2h_bytes_per_step": world * nbytes, "ms_per_step": e_ms, "steps": e_steps, "grids": grids,
               "what": "per step, all through the C ABI: sbp_set_state from pinned host memory (the 9-field "
                       f"state in the grid layout), sbp_step_n(1), sbp_get_state to pinned host memory{ranks}; "
                       f"{grids} grids on {grids} streams take the steps in turn (one grid's download, another's "
                       "upload and a step overlap)",
               "sequential_one_grid": {"value": rate(seq_ms), "ms_per_step": seq_ms, "steps": seq_steps}}
    elif math.isfinite(seq_ms):
        rec = {"value": rate(seq_ms), "unit": UNIT, "h2d_bytes_per_step": world * nbytes,
               "d2h_bytes_per_step": world * nbytes, "ms_per_step": seq_ms, "steps": seq_steps,
               "what": "per step, all through the C ABI on one grid: sbp_set_state from pinned host memory, "
                       f"sbp_step_n(1), sbp_get_state to pinned host memory (waited for){ranks}"}
    else:
        return {"value": None, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "error": note or "no end-to-end time"}
    if note:
        rec["note"] = note
    return rec


_BARRIER = None


def _pool_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def oracle_step_sample(sub, stages=5, j0=0):
    """Time the FP64 oracle on a sub-block (the top `sub` nodes of the workload's grid from r
    index j0, same map, medium and spacing): `stages` Runge-Kutta stages.  Returns (node-stages,
    seconds)."""
    import numpy as np

    from oracle import rk
    from oracle.elastic import Scheme, rhs
    from oracle.metrics import metrics
    from workloads.configs import config_by_name
    from workloads.fields import smooth_state
    from workloads.geometry import make_map
    from workloads.media import make_medium
    cfg = config_by_name(WORKLOAD)
    nq, nr, ns = cfg.nodes
    i, j, k = np.arange(sub[0]), np.arange(j0, j0 + sub[1]), np.arange(ns - sub[2], ns)
    fmap, fmed = make_map(cfg), make_medium(cfg)
    X = [np.broadcast_to(c, (sub[2], sub[1], sub[0])).copy()
         for c in fmap(i[None, None, :] / (nq - 1), j[None, :, None] / (nr - 1), k[:, None, None] / (ns - 1))]
    mat = fmed(*X)
    J, a = metrics(*X, cfg.order)
    sch = Scheme(cfg.order, sub)
    I, Jj, K = np.meshgrid(i, j, k, indexing="ij")
    Q = np.stack(smooth_state(cfg.nodes, 11, I.T, Jj.T, K.T))
    dQ = np.zeros_like(Q)
    if _BARRIER is not None:
        _BARRIER.wait(timeout=600)   # every core starts its timed stages together
    t0 = time.perf_counter()
    for s in range(stages):
        dQ *= rk.A[s]
        dQ += 1e-3 * rhs(Q, sch, J, a, mat, cfg.bc)
        Q += rk.B[s] * dQ
    return sub[0] * sub[1] * sub[2] * stages, time.perf_counter() - t0


def _oracle_worker(a):
    import os as _os
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        _os.environ[v] = "1"
    return oracle_step_sample(a[0], j0=a[1])


def host_cores():
    """Host cores available to this process and the CPU model (as /proc/cpuinfo names it)."""
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    model = ""
    try:
        for ln in open("/proc/cpuinfo"):
            k = ln.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware") and ":" in ln:
                model = ln.split(":", 1)[1].strip()
                break
            if k == "cpu part" and not model:
                model = "Arm part " + ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return n, (model or platform.processor() or platform.machine())


def oracle_parallel_sample(sub, nproc, repeats=1):
    """The oracle on nproc host cores at once: nproc spawned processes (one thread each), each
    timing one Runge-Kutta step on its own sub-block of the workload (the top `sub` nodes, at
    successive r offsets), after a barrier so that the timed stages run together.  Returns a
    list of (node-stages, seconds) per repeat: the node-stages of all cores and the slowest
    core's time."""
    import multiprocessing as mp
    jobs = [(sub, (w * sub[1]) % (1025 - sub[1])) for w in range(nproc)]
    ctx = mp.get_context("spawn")
    out = []
    with ctx.Pool(nproc, initializer=_pool_init, initargs=(ctx.Barrier(nproc),)) as pool:
        for _ in range(repeats):
            res = pool.map(_oracle_worker, jobs, chunksize=1)
            out.append((sum(r[0] for r in res), max(r[1] for r in res)))
    return out


REF_SUB = (257, 33, 17)     # per core and step of the reference arm
CPU_SUB = (1025, 33, 33)    # per core of the cpu_baseline


def run_reference(args, rank, world):
    if rank != 0:
        return
    sub = REF_SUB
    nproc, model = host_cores()
    runs = oracle_parallel_sample(sub, nproc, args.warmup + args.steps)[args.warmup:]
    tot = sum(t for _, t in runs)
    n_tot = sum(n for n, _ in runs)
    value = n_tot / tot / 1e6
    what = (f"per step, {nproc} spawned processes (one thread each) on {nproc} host cores ({model}), each one "
            f"5-stage RK step of the FP64 oracle on its own {sub[0]}x{sub[1]}x{sub[2]} block of the top of the "
            f"workload, started together after a barrier; time = the slowest core's")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": what, "nodes": list(sub), "order": 6},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "cpu_model": model, "kind": "oracle",
                         "sample": what},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# Adjoint stage, FP32 state: L^T and gradient 264 B (the metrics read once) + 80 B FP64 (rho, lambda,
# mu, J read, gradient read and written) + the prep (Wb_k = Wb + B_k Ub, yhat = H^-1 P~ Wb_k): on its
# own 156 B in one stage of five, fused into the previous stage's L^T pass (one more 36 B write) in
# the other four: 404 B per node and stage on average (sbp_adjoint_step); 384 B with the topography
# map's 4 metric fields (16 B, not 36).
ADJ_BYTES_PER_NODE_STAGE = 404
ADJ_BYTES_PER_NODE_STAGE_TOPO = 384


def run_adjoint(args, local):
    """One misfit gradient of the adjoint workload, timed on the device."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.adjoint import workload_problem
    from workloads.configs import config_by_name
    cfg = config_by_name("adjoint129_o4")
    nsteps = args.adj_steps or cfg.steps
    p, _, _ = workload_problem(cfg, 32, source_index="all", nsteps=nsteps)   # the eight sources, one batch
    s = p.s
    nq, nr, ns = cfg.nodes
    nodes = nq * nr * ns * p.B            # node-member pairs
    p.forward()                       # warm-up: one untimed forward run and gradient
    p.gradient()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    L.sbp_kernel_timing(s.h, True)
    L.sbp_kernel_times(s.h)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    phi = p.forward()
    ev[1].record(stream)
    g = p.gradient()
    ev[2].record(stream)
    torch.cuda.synchronize()
    kms, kn = L.sbp_kernel_times(s.h)
    L.sbp_kernel_timing(s.h, False)
    clk = clocks.stop()
    t_fwd, t_grad = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    adj_avg = kms[2] / max(1, kn[2])
    stage_avg = kms[0] / max(1, kn[0])
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    topo = s.map_path() == "topography"
    adj_bytes = ADJ_BYTES_PER_NODE_STAGE_TOPO if topo else ADJ_BYTES_PER_NODE_STAGE
    # the forward stage kernel's bytes, averaged over the five stages (stage 0 reads no RK register)
    stage_bytes = ((BYTES_PER_NODE_STAGE0_TOPO + 4 * BYTES_PER_NODE_STAGE_TOPO) / 5 if topo else
                   (BYTES_PER_NODE_STAGE0 + 4 * BYTES_PER_NODE_STAGE) / 5)
    achieved = adj_bytes * nodes / (adj_avg / 1e3) / 1e9
    value = nodes * 5 * nsteps / ((t_fwd + t_grad) / 1e3) / 1e6
    line = {
        "metric": "adjoint gradient throughput", "value": value, "unit": "Mnode-stage/s",
        "n_gpus": 1, "steps": nsteps, "warmup": nsteps, "ms_per_step": (t_fwd + t_grad) / nsteps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "adjoint129_o4", "nodes": list(cfg.nodes), "order": cfg.order,
                   "checkpoint_every": p.C, "receivers": len(p.receivers), "sources": p.B,
                   "batch": "the sources' states advance together (one launch per kernel)",
                   "warmup": "one untimed forward run and gradient over the same steps",
                   "l2": f"not flushed: each adjoint stage moves {adj_bytes * nodes / 1e9:.2f} GB, "
                         f"{adj_bytes * nodes / L2_BYTES:.0f} x L2",
                   "what": "node-stages of the forward problem (nodes x sources x 5 x steps) per second of "
                           "forward run + gradient"},
        "forward_ms": t_fwd, "gradient_ms": t_grad, "misfit": phi,
        "gradient_norm": float(g.double().norm()),
        "roofline": {"bound": "hbm", "achieved": achieved,
                     "kernel": "adjoint stage (gradient pass, L^T pass with the next stage's prep fused; "
                               "the prep alone in stage 4)",
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": adj_bytes * nodes, "algorithmic_bytes_per_node": adj_bytes,
                     "metric_path": "topography (a_q,x and a_s)" if topo else "general (9 metric fields)",
                     "avg_launch_ms": adj_avg, "launches": kn[2],
                     "peak_source": "measured" if peaks else "fallback"},
        "stage_kernel": {"avg_launch_ms": stage_avg, "launches": kn[0],
                         "achieved_gbs": stage_bytes * nodes / (stage_avg / 1e3) / 1e9,
                         "algorithmic_bytes_per_node_stage": stage_bytes},
        "kernel_ms": {"tiled": kms[0], "general": kms[1], "adjoint": kms[2], "launches": kn},
        "clocks": clk, "gpu_launches": int(kn[0] + kn[1] + 2 * kn[2]),
    }
    print(json.dumps(line), flush=True)


def run_surrogate_kernels(args, local):
    """The surrogate network's kernels at the surrogate workload's full size (3 inputs ->
    6 x 192 trace sets x 1024 samples, hidden 512, 128 channels): training iterations
    (forward, backward, Adam; batch 32) and the largest GEMM alone, against the BF16 peak."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300 import surrogate as S
    from paper_2011_02600_gb300.solver import _stream
    B = 32
    net = S.SurrogateNet(n_in=3, hidden=512, C=128, T0=32, n_up=5, n_out=192, seed=0)
    flops = [0]
    gemm = S.SurrogateNet._gemm

    def counting(M, N, K, *a, **k):
        flops[0] += 2 * M * N * K
        return gemm(M, N, K, *a, **k)
    net._gemm = counting
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.rand(3, B, generator=g).mul(2).sub(1).to(torch.bfloat16).cuda()
    m = torch.randn(6, B, generator=g).cuda()
    tgt = torch.randn(net.n_out, B * net.T, generator=g).cuda()

    def it():
        y = net.forward(x, m, keep=True)
        _, dy = S.mse(y, tgt)
        net.backward(dy)
        net.adam(1e-4)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    it_ms, it_flops, clk = None, None, None
    if not args.gemm_only:
        for _ in range(args.warmup):
            it()
        torch.cuda.synchronize()
        flops[0] = 0
        n_it = max(3, args.steps)
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        ev[0].record(stream)
        for _ in range(n_it):
            it()
        ev[1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        it_ms = ev[0].elapsed_time(ev[1]) / n_it
        it_flops = flops[0] / n_it
    # the largest GEMM alone: output layer forward, M = 6 x 192, N = B x 1024, K = 128 x 5, BF16
    # output (the six trace sets, stored like the network's other activations)
    M, N, K = net.n_last, B * net.T, net.C * 5
    A_ = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B_ = torch.randn(K, N, generator=g).to(torch.bfloat16).cuda()
    C_ = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
    def time_gemm(path, reps=20):
        """Device time of one GEMM: `reps` launches captured in a CUDA graph and replayed, so that
        the host's per-call work (argument marshalling) stays out of the measurement."""
        L.sbp_nn_set_gemm_path(path)
        for _ in range(3):   # warm-up: attributes set and operand tensor maps encoded
            L.sbp_nn_gemm(M, N, K, A_, K, 0, B_, N, 0, C_, N, 1, None, 0, 0.0, _stream())
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                L.sbp_nn_gemm(M, N, K, A_, K, 0, B_, N, 0, C_, N, 1, None, 0, 0.0, _stream())
        graph.replay()
        torch.cuda.synchronize()
        ev[0].record(stream)
        graph.replay()
        ev[1].record(stream)
        torch.cuda.synchronize()
        L.sbp_nn_set_gemm_path(0)
        return ev[0].elapsed_time(ev[1]) / reps
    g_ms = time_gemm(2)                  # tcgen05 kernel
    legacy_ms = time_gemm(1)             # mma.sync kernel, for comparison
    status = L.sbp_nn_status()
    tflops = 2.0 * M * N * K / (g_ms / 1e3) / 1e12
    peaks = _peaks()
    peak = peaks["bf16_tflops"] if peaks else 1900.0
    if args.gemm_only:   # the largest GEMM alone (profiling)
        print(json.dumps({"gemm_shape": [M, N, K], "avg_launch_ms": g_ms, "tflops": tflops, "status_bits": status}))
        return
    line = {
        "metric": "surrogate training iterations per second", "value": 1e3 / it_ms, "unit": "it/s",
        "n_gpus": 1, "steps": n_it, "warmup": args.warmup, "ms_per_step": it_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "clocks": clk,
        "data": "synthetic",
        "config": {"workload": "surrogate97_o4 network", "batch": B, "samples": net.T, "outputs": net.n_out,
                   "hidden": net.hidden, "channels": net.C, "params": net.n_params(),
                   "l2": (f"not flushed: the largest GEMM's operands and output ({(M * K + K * N + M * N) * 2 / 1e6:.0f}"
                          " MB) stay in L2 across the graph's back-to-back launches; the product is bound by the "
                          "tensor pipe, not by memory")},
        "ms_per_iteration": it_ms, "gemm_tflop_per_iteration": it_flops / 1e12,
        "gemm_tflops_in_iterations": it_flops / (it_ms / 1e3) / 1e12,
        "roofline": {"bound": "tensor", "kernel": "gemm_tc_kernel (TMA, tcgen05.mma kind::f16, TMEM accumulator, "
                               "BF16 output by TMA store)",
                     "shape": [M, N, K], "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": tflops / peak, "avg_launch_ms": g_ms, "status_bits": status,
                     "peak_source": "measured (cuBLAS bf16 burst)" if peaks else "fallback"},
        "legacy_mma_sync_gemm": {"avg_launch_ms": legacy_ms,
                                 "achieved_tflops": 2.0 * M * N * K / (legacy_ms / 1e3) / 1e12},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nodes", default=None,
                    help="nq,nr,ns: a smaller instance of the workload (same generators; for profiling)")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "adjoint129_o4", "surrogate97_o4"])
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--adj-steps", type=int, default=None, help="steps of the adjoint workload (default: its 1500)")
    ap.add_argument("--gemm-only", action="store_true",
                    help="surrogate workload: time only its largest GEMM (no training iterations; profiling)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "surrogate97_o4":
        if rank == 0:
            run_surrogate_kernels(args, local)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "adjoint129_o4":
        if rank == 0:
            run_adjoint(args, local)
        if dist:
            dist.destroy_process_group()
        return
    if args.warmup < 3:
        args.warmup = 3

    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_02600_gb300 import _lib as L
    from paper_2011_02600_gb300.solver import _stream
    from paper_2011_02600_gb300.workload_setup import build_solver
    from workloads.configs import config_by_name
    from workloads.fields import gaussian_pulse

    cfg = config_by_name(WORKLOAD)
    if args.nodes:
        import dataclasses
        cfg = dataclasses.replace(cfg, nodes=tuple(int(x) for x in args.nodes.split(",")))
    s, info = build_solver(cfg, precision=args.precision, device=f"cuda:{local}")
    elem = args.precision // 8
    nq, nr, ns = cfg.nodes
    nodes = nq * nr * ns
    dt = info["dt"]
    # initial state: a Gaussian velocity pulse at the centre of the block (timing workload)
    Lx, Ly, Lz = cfg.extent
    st = s.state()
    dev = s.device
    xs = torch.arange(nq, device=dev, dtype=torch.float64).view(1, 1, nq) * (Lx / (nq - 1))
    ys = torch.arange(nr, device=dev, dtype=torch.float64).view(1, nr, 1) * (Ly / (nr - 1))
    for k0 in range(0, ns, 32):
        k1 = min(ns, k0 + 32)
        zs = (-Lz + torch.arange(k0, k1, device=dev, dtype=torch.float64).view(-1, 1, 1) * (Lz / (ns - 1)))
        vals = gaussian_pulse(xs, ys, zs, (Lx / 2, Ly / 2, -Lz / 2), cfg.extra["pulse_width"], xp=torch)
        for f in range(9):
            st[f, k0:k1].copy_(vals[f].expand(k1 - k0, nr, nq))
    s.dq.zero_()
    stream = torch.cuda.current_stream()
    h = s.h
    for _ in range(args.warmup):
        L.sbp_step_n(h, 1, dt, _stream())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    L.sbp_kernel_timing(h, True)
    L.sbp_kernel_times(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        L.sbp_step_n(h, 1, dt, _stream())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kms, kn = L.sbp_kernel_times(h)
    L.sbp_kernel_timing(h, False)
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, dev)
    energy = s.energy()
    bits = s.status()
    ms_per_step = ms / args.steps
    value = world * nodes * 5 * args.steps / (ms / 1e3) / 1e6

    # the stage kernel (tiled unless the general path was selected) covers every node
    if kn[0] > 0:
        kind, launches, kms_tot, knodes = "tiled", kn[0], kms[0], nodes
    else:
        kind, launches, kms_tot, knodes = "general", kn[1], kms[1], nodes
    # per launch: stage 0 reads no RK register; average over the 5 stages of a step
    topo = kind == "tiled" and s.map_path() == "topography"
    b14, b0 = (BYTES_PER_NODE_STAGE_TOPO, BYTES_PER_NODE_STAGE0_TOPO) if topo else (BYTES_PER_NODE_STAGE,
                                                                                   BYTES_PER_NODE_STAGE0)
    flop_node = FLOP_PER_NODE_STAGE_TOPO if topo else FLOP_PER_NODE_STAGE
    avg_bytes = knodes * (b14 * 4 + b0) / 5.0 * (elem / 4)
    avg_ms = kms_tot / max(1, launches)
    achieved = avg_bytes / (avg_ms / 1e3) / 1e9
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    prof_traffic = None
    tpath = os.path.join(ROOT, "profiles", "stage_tiled_traffic.txt")
    if kind == "tiled" and os.path.exists(tpath):
        kv = {}
        for ln in open(tpath):
            if ":" in ln and not ln.startswith("#"):
                a, b2 = ln.split(":", 1)
                kv[a.strip()] = b2.strip()
        if kv.get("kernel_source_digest") == _kernel_digest() and \
                kv.get("metric_path", "general") == ("topography" if topo else "general"):
            per_node = (float(kv["dram_bytes_per_node_stage0"]) + 4 * float(kv["dram_bytes_per_node_stage1to4"])) / 5
            prof_traffic = per_node * knodes

    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": prof_traffic if elem == 4 else None, "kernel": kind,
            "algorithmic_bytes_per_launch": avg_bytes, "algorithmic_bytes_per_node_stage": [b0, b14],
            "metric_path": "topography (a_q,x and a_s)" if topo else "general (9 metric fields)",
            "avg_launch_ms": avg_ms,
            "launches": launches, "peak_source": "measured" if peaks else "fallback",
            "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS}
    if elem == 8:
        # FP64 is bound by the FP64 pipe, not by HBM: its peak is measured here by an FMA-chain probe
        fp64_peak = L.sbp_probe_fp64_rate(2000000, _stream())
        tflops = flop_node * knodes / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": tflops / fp64_peak, "traffic": None, "kernel": kind,
                "algorithmic_flop_per_launch": flop_node * knodes, "avg_launch_ms": avg_ms,
                "metric_path": "topography (a_q,x and a_s)" if topo else "general (9 metric fields)",
                "launches": launches,
                "peak_source": "measured: FP64 FMA-chain probe (sbp_probe_fp64_rate) on this device",
                "nominal_peak": FP64_NOMINAL_TFLOPS, "hbm_achieved_gbs": achieved, "hbm_frac": achieved / peak}

    # end to end through the C ABI: per step, a state uploaded from pinned host memory
    # (sbp_set_state), one RK step (sbp_step_n), the state downloaded to pinned host memory
    # (sbp_get_state).  Two or three grids on as many streams take the steps in turn, so that one
    # grid's download, another's upload and a step overlap (independent problems streamed through
    # the device); every step still moves its whole state in and out.  The same sequence on one
    # grid, each download waited for, is reported beside it.  Every rank runs this leg on its own
    # grids; the job's time is the slowest rank's, and the ranks on a node share its host memory.
    seq_ms, e_ms, ng, e_steps, note = None, None, 1, 0, None
    nbytes = 9 * s.fs * elem
    if dist:
        dist.barrier()   # every rank reads the free host memory before any of them pins some
    host_share = host_memory_share(int(os.environ.get("LOCAL_WORLD_SIZE", "1")))
    try:
        if host_share < 2 * 2 * nbytes:   # one pair of state buffers, with room to spare
            raise RuntimeError(f"{host_share / 1e9:.0f} GB of free host memory per rank: too little to pin "
                               f"two {nbytes / 1e9:.1f} GB state buffers")
        tdt = torch.float32 if elem == 4 else torch.float64
        host_in = [torch.empty(9 * s.fs, dtype=tdt, pin_memory=True)]
        host_out = [torch.empty(9 * s.fs, dtype=tdt, pin_memory=True)]
        for b in host_in + host_out:
            L.sbp_get_state(h, b, L.SBP_MEM_HOST, _stream())
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(args.e2e_steps):
            L.sbp_set_state(h, host_in[0], L.SBP_MEM_HOST, _stream())
            L.sbp_step_n(h, 1, dt, _stream())
            L.sbp_get_state(h, host_out[0], L.SBP_MEM_HOST, _stream())
        ev[1].record(stream)
        torch.cuda.synchronize()
        seq_ms = ev[0].elapsed_time(ev[1]) / args.e2e_steps
        # as many grids as fit (up to three): each stream's chain (upload, step, download) then
        # spans as many steps, and the copy engines and the SMs stay busy
        extra = []
        # a grid's fields (39) and its set-up buffers (coordinates, metrics and material in FP64: 16)
        footprint = (39 * elem + 16 * 8) * s.fs
        while len(extra) < 2:
            free, _total = torch.cuda.mem_get_info()
            if free < footprint:     # (a failed set-up below also stops here)
                break
            # host memory for this rank's pairs with the new one, and room for two more
            if host_share < (len(extra) + 4) * 2 * nbytes:
                break
            try:
                nb_in = torch.empty(9 * s.fs, dtype=tdt, pin_memory=True)
                nb_out = torch.empty(9 * s.fs, dtype=tdt, pin_memory=True)
            except Exception:
                break
            try:
                g2, _ = build_solver(cfg, precision=args.precision, device=f"cuda:{local}")
            except Exception:   # no room after all (the set-up's FP64 buffers): keep the grids so far
                del nb_in, nb_out
                torch.cuda.empty_cache()
                break
            L.sbp_get_state(g2.h, nb_in, L.SBP_MEM_HOST, _stream())
            L.sbp_get_state(g2.h, nb_out, L.SBP_MEM_HOST, _stream())
            extra.append(g2)
            host_in.append(nb_in)
            host_out.append(nb_out)
        if not extra:
            raise RuntimeError(f"no room for a second grid ({free / 1e9:.0f} GB free): sequential only")
        grids = [h] + [g2.h for g2 in extra]
        ng = len(grids)
        streams = [torch.cuda.Stream() for _ in range(ng)]
        nsteps = max(ng, ng * args.e2e_steps)

        def pipelined():
            start = torch.cuda.Event()
            start.record(stream)
            for st_ in streams:
                st_.wait_event(start)
            for n in range(nsteps):
                g, st_ = grids[n % ng], streams[n % ng]
                sp = st_.cuda_stream
                L.sbp_set_state(g, host_in[n % ng], L.SBP_MEM_HOST, sp)
                L.sbp_step_n(g, 1, dt, sp)
                L.sbp_get_state(g, host_out[n % ng], L.SBP_MEM_HOST | L.SBP_MEM_ASYNC, sp)
            for st_ in streams:
                done = torch.cuda.Event()
                done.record(st_)
                stream.wait_event(done)

        pipelined()  # warm-up of the added grids
        torch.cuda.synchronize()
        ev[0].record(stream)
        pipelined()
        ev[1].record(stream)
        torch.cuda.synchronize()
        e_ms = ev[0].elapsed_time(ev[1]) / nsteps
        e_steps = nsteps
        del host_in, host_out, extra
    except Exception as ex:  # pinned memory or a second grid's device memory can be unavailable
        note = str(ex)[:200]
        if e_ms is None:
            ng = 1
    # the job's times are the slowest rank's (a rank without a number counts as infinitely slow)
    seq_job = max_over_ranks(math.inf if seq_ms is None else seq_ms, dist, dev)
    e_job = max_over_ranks(math.inf if e_ms is None else e_ms, dist, dev)
    ng_job = -max_over_ranks(-ng, dist, dev)   # the fewest grids any rank streamed through
    e2e = e2e_record(nodes, world, nbytes, seq_job, e_job, int(ng_job), args.e2e_steps, e_steps, note)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sub = CPU_SUB
        nproc, model = host_cores()
        n, t = oracle_parallel_sample(sub, nproc)[0]
        cpu = {"value": n / t / 1e6, "unit": UNIT, "cores": nproc, "cpu_model": model, "kind": "oracle",
               "sample": f"{nproc} spawned processes (numpy/scipy, one thread each) on {nproc} host cores, each "
                         f"one 5-stage RK step of the FP64 oracle on its own {sub[0]}x{sub[1]}x{sub[2]} block of "
                         f"the top of the workload, started together after a barrier ({t:.1f} s, the slowest "
                         f"core's time)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if elem == 4 else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.nodes else WORKLOAD + " (reduced: profiling only)",
                   "nodes": list(cfg.nodes), "order": cfg.order,
                   "extent_m": list(cfg.extent), "stages_per_step": 5, "dt_s": dt,
                   "l2": (f"inputs larger than L2 (39 fields x {s.fs * elem / 1e9:.2f} GB resident)"
                          if 39 * s.fs * elem > L2_BYTES else
                          f"inputs smaller than L2 (39 fields x {s.fs * elem / 1e6:.1f} MB): reduced case"),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roof,
        "kernel_ms": {"tiled": kms[0], "general": kms[1], "launches": kn},
        "cpu_baseline": cpu,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": kn[0] + kn[1],
        "energy_after": energy, "status_bits": bits,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _kernel_digest():
    """Digest of the sources the stage kernel is built from (its translation unit, the
    headers it includes and the host code that encodes its tensor maps and launch shape)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2011_02600_gb300", "csrc")
    for f in ("kernels_tiled.cu", "tile_map.cuh", "common.cuh", "tma.cuh", "adjoint_terms.cuh", "sbp_coeffs.h",
              "launch.h", "adjoint_args.h", "api.cu"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
