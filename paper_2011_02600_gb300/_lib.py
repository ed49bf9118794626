"""ctypes binding of include/sbp.h: the same entry points, argument marshalling only.

Every function here forwards to the CUDA library libsbp_gb300.so and raises
SbpError on a non-zero status.  There is no CPU fallback: if the library is
not built, ``lib()`` raises.
"""
import ctypes
import os

from . import build as _build

SBP_BC_FREE = 0
SBP_BC_CHAR = 1
SBP_BC_INTERFACE = 2
SBP_TRADITIONAL = 100
SBP_MEM_HOST = 1
SBP_LAYOUT_DENSE = 2
SBP_MEM_ASYNC = 4
SBP_MAP_AUTO, SBP_MAP_GENERAL, SBP_MAP_TOPOGRAPHY = 0, 1, 2
ERRORS = {1: "ARG", 2: "UNSUPPORTED", 3: "CUDA", 4: "NONFINITE", 5: "STATE", 6: "MESH"}

EXPORTED = ("sbp_min_nodes", "sbp_create_grid", "sbp_destroy", "sbp_layout", "sbp_bind", "sbp_metrics",
            "sbp_set_material", "sbp_rhs", "sbp_rk_stage", "sbp_step_n", "sbp_set_kernel_path", "sbp_current",
            "sbp_kernel_timing", "sbp_kernel_times",
            "sbp_set_time", "sbp_get_time", "sbp_energy", "sbp_set_source", "sbp_set_receivers", "sbp_status",
            "sbp_rk_coefficients", "sbp_energy_noalloc", "sbp_rhs_adjoint", "sbp_adjoint_stage",
            "sbp_misfit", "sbp_set_batch", "sbp_set_sources", "sbp_nn_gemm", "sbp_nn_im2col", "sbp_nn_col2im",
            "sbp_nn_upsample2", "sbp_nn_relu_backward", "sbp_nn_bias_grad", "sbp_nn_mse", "sbp_nn_adam",
            "sbp_nn_mlp_to_conv", "sbp_nn_cast_bf16", "sbp_nn_moment_combine", "sbp_selftest_wait_timeout", "sbp_last_error",
            "sbp_set_receivers_xyz", "sbp_record_receivers", "sbp_set_state", "sbp_get_state",
            "sbp_nn_set_gemm_path", "sbp_nn_status", "sbp_set_slab", "sbp_interface_trace", "sbp_set_interface",
            "sbp_probe_fp64_rate", "sbp_set_map_path", "sbp_map_path", "sbp_adjoint_step",
            "sbp_nn_fourier_features")


class SbpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sbp error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class SbpGridDesc(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int32), ("nr", ctypes.c_int32), ("ns", ctypes.c_int32),
                ("order", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("bc_kind", ctypes.c_int32 * 6), ("bc_gamma", ctypes.c_double * 6)]


class SbpSource(ctypes.Structure):
    _fields_ = [("ref", ctypes.c_double * 3), ("moment", ctypes.c_double * 6), ("stf", ctypes.c_int32),
                ("f0", ctypes.c_double), ("t0", ctypes.c_double), ("T", ctypes.c_double)]


_LIB = None
P = ctypes.c_void_p


def lib(path=None):
    """Load the library (built by ``paper_2011_02600_gb300.build.build()``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2011_02600_gb300.build.build() "
                           "(this package has no CPU fallback)")
    L = ctypes.CDLL(path)
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sbp_min_nodes": [i32, ctypes.POINTER(i32)],
        "sbp_create_grid": [ctypes.POINTER(SbpGridDesc), ctypes.POINTER(P)],
        "sbp_destroy": [P],
        "sbp_layout": [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "sbp_bind": [P, P, P, P, P, P],
        "sbp_metrics": [P, P, P, P],
        "sbp_set_material": [P, P, P, P],
        "sbp_rhs": [P, P, P, P],
        "sbp_rk_stage": [P, i32, dbl, P],
        "sbp_step_n": [P, i32, dbl, P],
        "sbp_set_kernel_path": [P, i32],
        "sbp_set_map_path": [P, i32],
        "sbp_map_path": [P, ctypes.POINTER(i32)],
        "sbp_current": [P, ctypes.POINTER(i32)],
        "sbp_kernel_timing": [P, i32],
        "sbp_kernel_times": [P, ctypes.POINTER(dbl), ctypes.POINTER(i64)],
        "sbp_set_time": [P, dbl, i64],
        "sbp_get_time": [P, ctypes.POINTER(dbl), ctypes.POINTER(i64)],
        "sbp_energy": [P, ctypes.POINTER(dbl), P],
        "sbp_set_source": [P, ctypes.POINTER(SbpSource), P, P],
        "sbp_set_receivers": [P, i32, P, P, i32],
        "sbp_status": [P, ctypes.POINTER(ctypes.c_uint32), P],
        "sbp_rk_coefficients": [ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)],
        "sbp_energy_noalloc": [P, P, i32, i32, i32, i64, i64, i32, i32, i32, ctypes.POINTER(dbl), P],
        "sbp_rhs_adjoint": [P, P, P, P, P],
        "sbp_adjoint_stage": [P, i32, dbl, P, P, P, P, P, P, P],
        "sbp_adjoint_step": [P, dbl, P, P, P, P, P, P, P],
        "sbp_misfit": [P, P, P, dbl, P, P, P],
        "sbp_set_batch": [P, i32],
        "sbp_nn_gemm": [i32, i32, i32, P, i64, i32, P, i64, i32, P, i64, i32, P, i32, ctypes.c_float, P],
        "sbp_nn_im2col": [P, P, i32, i32, i32, i32, i32, P],
        "sbp_nn_col2im": [P, P, i32, i32, i32, i32, i32, P],
        "sbp_nn_upsample2": [P, P, i64, i32, i32, P],
        "sbp_nn_relu_backward": [P, P, P, i64, P],
        "sbp_nn_bias_grad": [P, P, i32, i64, P],
        "sbp_nn_mse": [P, P, P, i64, P, i32, P],
        "sbp_nn_adam": [P, P, P, P, P, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32, P],
        "sbp_nn_mlp_to_conv": [P, P, i32, i32, i32, i32, P],
        "sbp_nn_cast_bf16": [P, P, i64, P],
        "sbp_nn_fourier_features": [P, P, i32, i64, i32, P],
        "sbp_nn_moment_combine": [P, P, P, P, P, i32, i32, i32, i32, P],
        "sbp_selftest_wait_timeout": [P, ctypes.c_uint32, P],
        "sbp_set_sources": [P, i32, ctypes.POINTER(SbpSource), P, P],
        "sbp_set_receivers_xyz": [P, i32, P, P, i32, P, i32, P],
        "sbp_record_receivers": [P, P, i32, P],
        "sbp_set_state": [P, P, i32, P],
        "sbp_get_state": [P, P, i32, P],
        "sbp_nn_set_gemm_path": [i32],
        "sbp_nn_status": [ctypes.POINTER(ctypes.c_uint32)],
        "sbp_set_slab": [P, i32, i32, i32, i32],
        "sbp_interface_trace": [P, i32, P, P, P],
        "sbp_set_interface": [P, i32, P],
        "sbp_probe_fp64_rate": [i32, ctypes.POINTER(dbl), P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.sbp_last_error.argtypes = []
    L.sbp_last_error.restype = ctypes.c_char_p
    _LIB = L
    return L


def _check(rc):
    if rc != 0:
        raise SbpError(rc, lib().sbp_last_error().decode())


def _ptr(x):
    """Device/host pointer of a torch tensor, an int address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def sbp_min_nodes(order):
    out = ctypes.c_int32()
    _check(lib().sbp_min_nodes(order, ctypes.byref(out)))
    return out.value


def sbp_create_grid(nodes, order, precision, bc):
    """bc: six entries ("free",) or ("char", gamma), faces (q0, q1, r0, r1, s0, s1)."""
    d = SbpGridDesc()
    d.nq, d.nr, d.ns = nodes
    d.order, d.precision = order, precision
    for f, c in enumerate(bc):
        d.bc_kind[f] = {"free": SBP_BC_FREE, "char": SBP_BC_CHAR, "interface": SBP_BC_INTERFACE}[c[0]]
        d.bc_gamma[f] = float(c[1]) if c[0] == "char" else 0.0
    h = P()
    _check(lib().sbp_create_grid(ctypes.byref(d), ctypes.byref(h)))
    return h


def sbp_destroy(h):
    _check(lib().sbp_destroy(h))


def sbp_layout(h):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sbp_layout(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sbp_bind(h, q0, q1, dq, met, mat):
    _check(lib().sbp_bind(h, _ptr(q0), _ptr(q1), _ptr(dq), _ptr(met), _ptr(mat)))


def sbp_metrics(h, xyz, jmet, stream):
    _check(lib().sbp_metrics(h, _ptr(xyz), _ptr(jmet), stream))


def sbp_set_material(h, jmet, rlm, stream):
    _check(lib().sbp_set_material(h, _ptr(jmet), _ptr(rlm), stream))


def sbp_rhs(h, q, out, stream):
    _check(lib().sbp_rhs(h, _ptr(q), _ptr(out), stream))


def sbp_rk_stage(h, stage, dt, stream):
    _check(lib().sbp_rk_stage(h, stage, dt, stream))


def sbp_step_n(h, n, dt, stream):
    _check(lib().sbp_step_n(h, n, dt, stream))


def sbp_set_kernel_path(h, path):
    _check(lib().sbp_set_kernel_path(h, path))


def sbp_set_map_path(h, path):
    _check(lib().sbp_set_map_path(h, path))


def sbp_map_path(h):
    v = ctypes.c_int32(0)
    _check(lib().sbp_map_path(h, ctypes.byref(v)))
    return v.value


def sbp_kernel_timing(h, enable):
    _check(lib().sbp_kernel_timing(h, 1 if enable else 0))


def sbp_kernel_times(h):
    """([ms_tiled, ms_general, ms_adjoint], [launches ...]) since the previous call."""
    ms, n = (ctypes.c_double * 3)(), (ctypes.c_int64 * 3)()
    _check(lib().sbp_kernel_times(h, ms, n))
    return list(ms), list(n)


def sbp_current(h):
    w = ctypes.c_int32()
    _check(lib().sbp_current(h, ctypes.byref(w)))
    return w.value


def sbp_set_time(h, t, step):
    _check(lib().sbp_set_time(h, t, step))


def sbp_get_time(h):
    t, s = ctypes.c_double(), ctypes.c_int64()
    _check(lib().sbp_get_time(h, ctypes.byref(t), ctypes.byref(s)))
    return t.value, s.value


def sbp_energy(h, stream):
    out = ctypes.c_double()
    _check(lib().sbp_energy(h, ctypes.byref(out), stream))
    return out.value


def sbp_set_source(h, ref, moment, stf, f0, t0, T, jmet, stream):
    s = SbpSource()
    for a in range(3):
        s.ref[a] = ref[a]
    for c in range(6):
        s.moment[c] = moment[c]
    s.stf, s.f0, s.t0, s.T = stf, f0, t0, T
    _check(lib().sbp_set_source(h, ctypes.byref(s), _ptr(jmet), stream))


def sbp_set_receivers(h, ijk, traces, n_t):
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
    _check(lib().sbp_set_receivers(h, len(arr), arr.ctypes.data if len(arr) else None, _ptr(traces), n_t))


def sbp_set_receivers_xyz(h, xyz, coords, face, traces, n_t):
    """Receivers at the nodes nearest to host points xyz (n x 3); returns the chosen (i, j, k)."""
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    ijk = np.zeros((len(arr), 3), dtype=np.int32)
    _check(lib().sbp_set_receivers_xyz(h, len(arr), arr.ctypes.data if len(arr) else None, _ptr(coords), face,
                                       _ptr(traces), n_t, ijk.ctypes.data if len(arr) else None))
    return ijk


def _buf(x):
    """Pointer of a torch tensor or a numpy array (host memory)."""
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return _ptr(x)


def sbp_record_receivers(h, dst, flags, stream):
    _check(lib().sbp_record_receivers(h, _buf(dst), flags, stream))


def sbp_set_state(h, src, flags, stream):
    _check(lib().sbp_set_state(h, _buf(src), flags, stream))


def sbp_get_state(h, dst, flags, stream):
    _check(lib().sbp_get_state(h, _buf(dst), flags, stream))


def sbp_status(h, stream):
    v = ctypes.c_uint32()
    _check(lib().sbp_status(h, ctypes.byref(v), stream))
    return v.value


def sbp_rk_coefficients():
    A, B, C = (ctypes.c_double * 5)(), (ctypes.c_double * 5)(), (ctypes.c_double * 5)()
    _check(lib().sbp_rk_coefficients(A, B, C))
    return list(A), list(B), list(C)


def sbp_energy_noalloc(q, mat, nodes, ldq, fs, order, precision, nblocks, stream):
    """Energy from plain device pointers, with the library's static scratch (no allocation)."""
    out = ctypes.c_double()
    nq, nr, ns = nodes
    _check(lib().sbp_energy_noalloc(_ptr(q), _ptr(mat), nq, nr, ns, ldq, fs, order, precision, nblocks,
                                    ctypes.byref(out), stream))
    return out.value


def sbp_rhs_adjoint(h, w, out, scratch, stream):
    _check(lib().sbp_rhs_adjoint(h, _ptr(w), _ptr(out), _ptr(scratch), stream))


def sbp_adjoint_step(h, dt, u_stages, ubar, wbar, scratch, rlmj, grad, stream):
    _check(lib().sbp_adjoint_step(h, dt, _ptr(u_stages), _ptr(ubar), _ptr(wbar), _ptr(scratch), _ptr(rlmj),
                                  _ptr(grad), stream))


def sbp_adjoint_stage(h, stage, dt, u_stage, ubar, wbar, scratch, rlmj, grad, stream):
    _check(lib().sbp_adjoint_stage(h, stage, dt, _ptr(u_stage), _ptr(ubar), _ptr(wbar), _ptr(scratch),
                                   _ptr(rlmj), _ptr(grad), stream))


def sbp_misfit(h, q, data, weight, acc, ubar, stream):
    _check(lib().sbp_misfit(h, _ptr(q), _ptr(data), weight, _ptr(acc), _ptr(ubar), stream))


def sbp_set_slab(h, ns_global, k_offset, ghost_lo, ghost_hi):
    _check(lib().sbp_set_slab(h, ns_global, k_offset, ghost_lo, ghost_hi))


def sbp_interface_trace(h, face, q, trace, stream):
    _check(lib().sbp_interface_trace(h, face, _ptr(q), _ptr(trace), stream))


def sbp_set_interface(h, face, other_trace):
    _check(lib().sbp_set_interface(h, face, _ptr(other_trace)))


def sbp_probe_fp64_rate(iters, stream):
    out = ctypes.c_double()
    _check(lib().sbp_probe_fp64_rate(iters, ctypes.byref(out), stream))
    return out.value


def sbp_set_batch(h, nb):
    _check(lib().sbp_set_batch(h, nb))


def sbp_set_sources(h, sources, jmet, stream):
    """sources: list of dicts with ref, moment, stf (0/1), f0, t0, T."""
    arr = (SbpSource * max(1, len(sources)))()
    for m, src in enumerate(sources):
        for a in range(3):
            arr[m].ref[a] = src["ref"][a]
        for c in range(6):
            arr[m].moment[c] = src["moment"][c]
        arr[m].stf, arr[m].f0, arr[m].t0, arr[m].T = src["stf"], src["f0"], src["t0"], src.get("T", 0.1)
    _check(lib().sbp_set_sources(h, len(sources), arr, _ptr(jmet), stream))


def sbp_nn_gemm(M, N, K, A, lda, transA, B, ldb, transB, C, ldc, c_bf16, bias, relu, beta, stream):
    _check(lib().sbp_nn_gemm(M, N, K, _ptr(A), lda, transA, _ptr(B), ldb, transB, _ptr(C), ldc, c_bf16, _ptr(bias),
                             relu, beta, stream))


def sbp_nn_set_gemm_path(path):
    _check(lib().sbp_nn_set_gemm_path(path))


def sbp_nn_status():
    v = ctypes.c_uint32()
    _check(lib().sbp_nn_status(ctypes.byref(v)))
    return v.value


def sbp_nn_im2col(X, Xc, C, B, T, kw, pad, stream):
    _check(lib().sbp_nn_im2col(_ptr(X), _ptr(Xc), C, B, T, kw, pad, stream))


def sbp_nn_col2im(dXc, dX, C, B, T, kw, pad, stream):
    _check(lib().sbp_nn_col2im(_ptr(dXc), _ptr(dX), C, B, T, kw, pad, stream))


def sbp_nn_upsample2(X, Y, rows, T, backward, stream):
    _check(lib().sbp_nn_upsample2(_ptr(X), _ptr(Y), rows, T, backward, stream))


def sbp_nn_relu_backward(dA, A, dZ, n, stream):
    _check(lib().sbp_nn_relu_backward(_ptr(dA), _ptr(A), _ptr(dZ), n, stream))


def sbp_nn_bias_grad(dZ, db, M, N, stream):
    _check(lib().sbp_nn_bias_grad(_ptr(dZ), _ptr(db), M, N, stream))


def sbp_nn_mse(Y, Tg, dY, n, partial, nblocks, stream):
    _check(lib().sbp_nn_mse(_ptr(Y), _ptr(Tg), _ptr(dY), n, _ptr(partial), nblocks, stream))


def sbp_nn_adam(w, g, m, v, w_bf16, n, lr, b1, b2, eps, step, stream):
    _check(lib().sbp_nn_adam(_ptr(w), _ptr(g), _ptr(m), _ptr(v), _ptr(w_bf16), n, lr, b1, b2, eps, step, stream))


def sbp_nn_mlp_to_conv(H, X, C, T0, B, backward, stream):
    _check(lib().sbp_nn_mlp_to_conv(_ptr(H), _ptr(X), C, T0, B, backward, stream))


def sbp_nn_cast_bf16(x, y, n, stream):
    _check(lib().sbp_nn_cast_bf16(_ptr(x), _ptr(y), n, stream))


def sbp_nn_fourier_features(x, y, n_in, B, L, stream):
    _check(lib().sbp_nn_fourier_features(_ptr(x), _ptr(y), n_in, B, L, stream))


def sbp_nn_moment_combine(G, m, y, dy, dG, n_out, B, T, backward, stream):
    _check(lib().sbp_nn_moment_combine(_ptr(G), _ptr(m), _ptr(y), _ptr(dy), _ptr(dG), n_out, B, T, backward, stream))


def sbp_selftest_wait_timeout(h, polls, stream):
    _check(lib().sbp_selftest_wait_timeout(h, polls, stream))
