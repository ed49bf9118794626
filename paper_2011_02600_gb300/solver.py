"""Torch-backed convenience layer over the C ABI: device buffers and streams.

PyTorch provides device memory and the current CUDA stream; every step of the
scheme runs in the library's kernels.
"""
import torch

from . import _lib as L

FACES = ("q0", "q1", "r0", "r1", "s0", "s1")


def _stream():
    return ctypes_stream(torch.cuda.current_stream())


def ctypes_stream(s):
    return s.cuda_stream


def _on_host(x):
    """True for numpy arrays and CPU tensors."""
    return not isinstance(x, torch.Tensor) or x.device.type == "cpu"


class ElasticSolver:
    """One curvilinear block on one GPU.

    nodes = (nq, nr, ns); order: 2..7 for the upwind pairs of Table 1, 2, 4 or 6 with
    operator="traditional" for the central operators of Table 2; precision in {32, 64};
    bc: six face conditions ("free",) / ("char", gamma); slab: (ns of the whole block,
    k_offset, ghost_lo, ghost_hi) when the grid is one s-slab of a decomposed block (slab.py).
    """

    def __init__(self, nodes, order, precision=32, bc=None, device="cuda", batch=1, operator="upwind", slab=None):
        if bc is None:
            bc = [("char", 0.0)] * 5 + [("free",)]
        if operator not in ("upwind", "traditional"):
            raise ValueError(f"unknown operator family {operator!r}")
        self.nodes = tuple(int(n) for n in nodes)
        self.order = order
        self.operator = operator
        self.code = order + (L.SBP_TRADITIONAL if operator == "traditional" else 0)
        self.precision = precision
        self.bc = list(bc)
        self.device = torch.device(device)
        self.dtype = torch.float32 if precision == 32 else torch.float64
        self.h = L.sbp_create_grid(self.nodes, self.code, precision, self.bc)
        self.batch = int(batch)
        if self.batch != 1:
            L.sbp_set_batch(self.h, self.batch)
        if slab is not None:   # (ns of the block, k_offset, ghost_lo, ghost_hi): see slab.py
            L.sbp_set_slab(self.h, *slab)
        self.ldq, self.fs, self.elem = L.sbp_layout(self.h)
        kw = dict(dtype=self.dtype, device=self.device)
        nst = 9 * self.batch
        self.qbuf = [torch.zeros(nst * self.fs, **kw), torch.zeros(nst * self.fs, **kw)]
        self.dq = torch.zeros(nst * self.fs, **kw)
        self.met = torch.zeros(9 * self.fs, **kw)
        self.mat = torch.zeros(3 * self.fs, **kw)
        L.sbp_bind(self.h, self.qbuf[0], self.qbuf[1], self.dq, self.met, self.mat)
        self.jmet = None
        self.traces = None

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                L.sbp_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # -- layout helpers -------------------------------------------------------
    def view(self, flat, nf):
        """(nf, ns, nr, nq) strided view of a flat buffer in the library layout."""
        nq, nr, ns = self.nodes
        return flat[: nf * self.fs].view(nf, self.fs)[:, : ns * nr * self.ldq].view(nf, ns, nr, self.ldq)[..., :nq]

    def new_fields(self, nf, dtype=None):
        return torch.zeros(nf * self.fs, dtype=dtype or self.dtype, device=self.device)

    def to_layout(self, arr, dtype=None):
        """Copy an (nf, ns, nr, nq) tensor into a fresh flat buffer in the library layout."""
        nf = arr.shape[0]
        buf = self.new_fields(nf, dtype or arr.dtype)
        self.view(buf, nf).copy_(arr.to(device=self.device, dtype=buf.dtype))
        return buf

    # -- setup ----------------------------------------------------------------
    def setup(self, xyz, rlm, keep_metrics=False):
        """xyz: (3, ns, nr, nq) coordinates; rlm: (3, ns, nr, nq) rho, lambda, mu (FP64 or castable)."""
        st = _stream()
        xyz_b = self.to_layout(torch.as_tensor(xyz), torch.float64)
        jmet = self.new_fields(10, torch.float64)
        L.sbp_metrics(self.h, xyz_b, jmet, st)
        del xyz_b
        rlm_b = self.to_layout(torch.as_tensor(rlm), torch.float64)
        L.sbp_set_material(self.h, jmet, rlm_b, st)
        del rlm_b
        bits = L.sbp_status(self.h, st)
        if bits & 2:
            raise L.SbpError(6, "non-positive Jacobian")
        if bits & 4:
            raise L.SbpError(6, "invalid material (rho, mu > 0 and lambda + 2 mu > 0 required)")
        self.jmet = jmet if keep_metrics else None
        return jmet

    def metrics(self):
        """(J, a) as (ns, nr, nq) and (3, 3, ns, nr, nq) views of the FP64 metric buffer."""
        v = self.view(self.jmet, 10)
        return v[0], v[1:].reshape(3, 3, *v.shape[1:])

    # -- state ------------------------------------------------------------------
    @property
    def current(self):
        return L.sbp_current(self.h)

    def state(self, member=0):
        """(9, ns, nr, nq) view of the current state (of batch member `member`)."""
        return self.view(self.qbuf[self.current][member * 9 * self.fs:], 9)

    def set_state(self, Q, reset_register=True):
        self.state().copy_(torch.as_tensor(Q).to(device=self.device, dtype=self.dtype))
        if reset_register:
            self.dq.zero_()

    def set_time(self, t, step=0):
        L.sbp_set_time(self.h, t, step)

    @property
    def time(self):
        return L.sbp_get_time(self.h)[0]

    def set_kernel_path(self, path):
        L.sbp_set_kernel_path(self.h, path)

    def set_map_path(self, path):
        """"auto" (the topography path where the metrics allow it) or "general"."""
        L.sbp_set_map_path(self.h, {"auto": L.SBP_MAP_AUTO, "general": L.SBP_MAP_GENERAL}[path])

    def map_path(self):
        """The metric path of the tiled forward stage: "topography" or "general"."""
        return "topography" if L.sbp_map_path(self.h) == L.SBP_MAP_TOPOGRAPHY else "general"

    # -- compute ----------------------------------------------------------------
    def rhs(self, Q=None):
        """dQ/dt (9, ns, nr, nq) of the given state (default: the current one)."""
        src = self.qbuf[self.current] if Q is None else self.to_layout(torch.as_tensor(Q), self.dtype)
        out = self.new_fields(9)
        L.sbp_rhs(self.h, src, out, _stream())
        return self.view(out, 9)

    def rk_stage(self, k, dt):
        L.sbp_rk_stage(self.h, k, dt, _stream())

    def step(self, n, dt, check_every=0):
        """n Runge-Kutta steps of size dt.  With check_every = m > 0 the discrete energy is
        formed every m steps and a non-finite state raises SbpError (SBP_ERR_NONFINITE, code 4)
        before further steps run (the check covers the first batch member)."""
        if check_every <= 0:
            L.sbp_step_n(self.h, n, dt, _stream())
            return
        done = 0
        while done < n:
            k = min(int(check_every), n - done)
            L.sbp_step_n(self.h, k, dt, _stream())
            done += k
            self.energy()

    def save_state(self, path):
        """Write the state, the Runge-Kutta register, the time and the step counter to path
        (between steps; see checkpoint.py for the format)."""
        from . import checkpoint
        t, step = L.sbp_get_time(self.h)
        header = dict(nodes=list(self.nodes), order=self.code, precision=self.precision, batch=self.batch,
                      ldq=self.ldq, fs=self.fs, time=t, step=step)
        data = checkpoint.pack(header, [self.qbuf[self.current].cpu().numpy(), self.dq.cpu().numpy()])
        with open(path, "wb") as f:
            f.write(data)

    def load_state(self, path):
        """Resume from a file written by save_state on a grid of the same shape, order,
        precision, batch and layout (checkpoint.CheckpointError otherwise)."""
        from . import checkpoint
        with open(path, "rb") as f:
            header, (q, dq) = checkpoint.unpack(f.read())
        want = dict(nodes=list(self.nodes), order=self.code, precision=self.precision, batch=self.batch,
                    ldq=self.ldq, fs=self.fs)
        for k, v in want.items():
            if header.get(k) != v:
                raise checkpoint.CheckpointError(f"checkpoint {k} {header.get(k)} does not match the grid's {v}")
        if q.size != self.qbuf[0].numel() or dq.size != self.dq.numel():
            raise checkpoint.CheckpointError("checkpoint array sizes do not match the grid")
        self.qbuf[self.current].copy_(torch.from_numpy(q))
        self.dq.copy_(torch.from_numpy(dq))
        L.sbp_set_time(self.h, float(header["time"]), int(header["step"]))

    def energy(self):
        return L.sbp_energy(self.h, _stream())

    def status(self):
        return L.sbp_status(self.h, _stream())

    def set_source(self, ref, moment, stf="ricker", f0=2.0, t0=None, T=0.1):
        if self.jmet is None:
            raise RuntimeError("set_source needs setup(..., keep_metrics=True)")
        kind = 0 if stf == "ricker" else 1
        L.sbp_set_source(self.h, ref, moment, kind, f0, 1.2 / f0 if t0 is None else t0, T, self.jmet, _stream())

    def set_sources(self, sources, f0=2.0, t0=None):
        """One Ricker point source per batch member: dicts with ref (q, r, s) and moment (Voigt)."""
        if self.jmet is None:
            raise RuntimeError("set_sources needs setup(..., keep_metrics=True)")
        t0 = 1.2 / f0 if t0 is None else t0
        L.sbp_set_sources(self.h, [dict(ref=sc["ref"], moment=sc["moment"], stf=0, f0=f0, t0=t0) for sc in sources],
                          self.jmet, _stream())

    def upload_state(self, src, dense=True):
        """Copy the current state in from a host numpy array or a torch tensor (host or device):
        [B * 9][ns][nr][nq] packed when dense, else the flat grid layout (sbp_set_state)."""
        flags = (L.SBP_LAYOUT_DENSE if dense else 0) | (L.SBP_MEM_HOST if _on_host(src) else 0)
        L.sbp_set_state(self.h, src, flags, _stream())

    def download_state(self, dst, dense=True):
        """Copy the current state out to dst (host numpy array or torch tensor; sbp_get_state)."""
        flags = (L.SBP_LAYOUT_DENSE if dense else 0) | (L.SBP_MEM_HOST if _on_host(dst) else 0)
        L.sbp_get_state(self.h, dst, flags, _stream())
        return dst

    def set_receivers_at(self, points, coords, n_t, face=5):
        """Receivers at the nodes nearest to the physical points (n x 3), searched on face `face`
        (5: the top surface s = 1; -1: every node) of the node coordinates coords (3, ns, nr, nq).
        The library keeps the traces (read them with record_receivers).  Returns the chosen
        (i, j, k) per receiver."""
        xyz_b = self.to_layout(torch.as_tensor(coords), torch.float64)
        ijk = L.sbp_set_receivers_xyz(self.h, points, xyz_b, face, None, n_t)
        self.traces = None
        self._rec_shape = (len(ijk), n_t)
        return ijk

    def record_receivers(self, host=True):
        """The traces recorded so far: [B][n][3][n_t] (without the batch axis when B = 1), a host
        numpy array (host=True) or a device tensor."""
        import numpy as np
        n, n_t = self._rec_shape
        shape = (self.batch, n, 3, n_t)
        if host:
            out = np.zeros(shape, dtype=np.float32 if self.precision == 32 else np.float64)
            L.sbp_record_receivers(self.h, out, L.SBP_MEM_HOST, _stream())
        else:
            out = torch.zeros(shape, dtype=self.dtype, device=self.device)
            L.sbp_record_receivers(self.h, out, 0, _stream())
        return out if self.batch > 1 else out[0]

    def set_receivers(self, ijk, n_t):
        """Traces view [member][receiver][component][step] (the member axis only when batched)."""
        n = len(ijk)
        self.traces = torch.zeros(self.batch * max(n, 1) * 3 * n_t, dtype=self.dtype, device=self.device)
        L.sbp_set_receivers(self.h, ijk, self.traces, n_t)
        self._rec_shape = (n, n_t)
        tr = self.traces.view(self.batch, -1, 3, n_t)[:, :n]
        return tr if self.batch > 1 else tr[0]

