"""The kernels' per-node operator on the CPU: tests/host_operator.cpp compiles raw_operator_at and
apply_P of csrc/common.cuh (rows of D+ and D-, flux and strain forms, free-surface and
characteristic penalties, P~) as host C++; its dQ/dt at every node of a curvilinear grid with a
random medium and a random state is compared with the oracle's right-hand side (Eq.
gen_hyp_transformed_discrete_SAT) in FP64.  The metric terms are inputs here (the oracle's,
Sec. 2.2); the stored coefficients 1/(rho J), lambda/J, mu/J are formed as the library forms
them.  Orders 2 to 7: the kernels are launched for 2, 4 and 6, and the odd orders' tables and
rows are checked here ahead of their GPU runs."""
import ctypes

import numpy as np
import pytest

from oracle.elastic import Scheme, energy, rhs
from oracle.metrics import metrics
from workloads.fields import random_state, smooth_state
from workloads.geometry import make_map, node_coordinates
from workloads.media import make_medium

from host_build import build

BCS = {
    "free": [("free",)] * 6,
    "char": [("char", g) for g in (0.0, 0.3, -0.4, 1.0, -1.0, 0.25)],
    "mixed": [("char", 0.0), ("free",), ("char", 0.6), ("free",), ("char", -0.2), ("free",)],
}


@pytest.fixture(scope="module")
def hostop(tmp_path_factory):
    so = build("host_operator.cpp", tmp_path_factory.mktemp("hostop") / "libhostop.so", shared=True)
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    for fn in (lib.host_rhs, lib.host_rhs_f32):
        fn.argtypes = [ctypes.c_int] * 4 + [P] * 6
        fn.restype = ctypes.c_int
    lib.host_energy.argtypes = [ctypes.c_int] * 4 + [P] * 3
    lib.host_energy.restype = ctypes.c_int
    lib.host_metrics.argtypes = [ctypes.c_int] * 4 + [P] * 2
    lib.host_metrics.restype = ctypes.c_longlong
    lib.host_delta_1d.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P]
    lib.host_delta_1d.restype = ctypes.c_int
    return lib


def _host_rhs(lib, order, Q, J, a, mat, bc, dtype=np.float64):
    """dQ/dt of the host-compiled kernel operator; FP32 arrays (state, metrics, coefficients cast
    from FP64 as the library stores them) when dtype is float32."""
    ns, nr, nq = J.shape
    rho, lam, mu = mat
    met = np.ascontiguousarray(np.stack([a[xi][c] for xi in range(3) for c in range(3)]).astype(dtype))
    coef = np.ascontiguousarray(np.stack([1.0 / (rho * J), lam / J, mu / J]).astype(dtype))
    q = np.ascontiguousarray(np.asarray(Q).astype(dtype))
    kind = (ctypes.c_int * 6)(*[0 if b[0] == "free" else 1 for b in bc])
    gamma = (ctypes.c_double * 6)(*[0.0 if b[0] == "free" else b[1] for b in bc])
    out = np.empty_like(q)
    fn = lib.host_rhs if dtype == np.float64 else lib.host_rhs_f32
    rc = fn(order, nq, nr, ns, q.ctypes.data, met.ctypes.data, coef.ctypes.data,
            ctypes.cast(kind, ctypes.c_void_p), ctypes.cast(gamma, ctypes.c_void_p), out.ctypes.data)
    assert rc == 0
    return out


@pytest.mark.parametrize("order,nodes", [(2, (9, 7, 8)), (3, (8, 9, 7)), (4, (13, 12, 14)), (5, (12, 13, 11)), (6, (18, 16, 17)),
                                         (7, (17, 18, 16))])
@pytest.mark.parametrize("bcname", sorted(BCS))
def test_kernel_operator_matches_oracle_fp64(hostop, order, nodes, bcname):
    bc = BCS[bcname]
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    J, a = metrics(*X, order)
    rng = np.random.default_rng(order * 10 + len(bcname))
    shape = J.shape
    rho = rng.uniform(2000.0, 3000.0, shape)
    mu = rho * rng.uniform(1500.0, 3000.0, shape) ** 2
    lam = rho * rng.uniform(3000.0, 6000.0, shape) ** 2 - 2 * mu
    lam = np.maximum(lam, 0.1 * mu)
    mat = (rho, lam, mu)
    Q = random_state(nodes, 21 + order, 1.0, 1.0e6)
    got = _host_rhs(hostop, order, Q, J, a, mat, bc)
    want = rhs(Q, Scheme(order, nodes), J, a, mat, bc)
    err = np.abs(got - want).max(axis=(1, 2, 3)) / np.abs(want).max(axis=(1, 2, 3))
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("order,nodes", [(2, (9, 7, 8)), (3, (8, 9, 7)), (4, (13, 12, 14)), (5, (12, 13, 11)), (6, (18, 16, 17)),
                                         (7, (17, 18, 16))])
@pytest.mark.parametrize("bcname", sorted(BCS))
def test_kernel_operator_matches_oracle_fp32(hostop, order, nodes, bcname):
    """The FP32 instantiation (FP32 closure tables, weights and penalty arithmetic) on a smooth
    state, within the FP32 tolerance of the GPU parity tests (5e-5 of each field's peak)."""
    bc = BCS[bcname]
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    J, a = metrics(*X, order)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    K, Jj, I = np.meshgrid(np.arange(nodes[2]), np.arange(nodes[1]), np.arange(nodes[0]), indexing="ij")
    Q = np.stack(smooth_state(nodes, 9, I, Jj, K))
    got = _host_rhs(hostop, order, Q, J, a, mat, bc, np.float32)
    want = rhs(Q, Scheme(order, nodes), J, a, mat, bc)
    err = np.abs(got - want).max(axis=(1, 2, 3)) / np.abs(want).max(axis=(1, 2, 3))
    assert err.max() < 5e-5, err


@pytest.mark.parametrize("order,nodes", [(2, (9, 7, 8)), (3, (8, 9, 7)), (4, (13, 12, 14)), (5, (12, 13, 11)), (6, (18, 16, 17)),
                                         (7, (17, 18, 16))])
def test_kernel_energy_density_matches_oracle(hostop, order, nodes):
    """The energy kernel's per-node density (one division, from the stored 1/(rho J), lambda/J,
    mu/J) and norm weights give the oracle's discrete energy (Eq. physical_energy_discrete with
    P~) to rounding, for a random state and medium on a curvilinear grid."""
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    J, a = metrics(*X, order)
    rng = np.random.default_rng(order)
    rho = rng.uniform(2000.0, 3000.0, J.shape)
    mu = rho * rng.uniform(1500.0, 3000.0, J.shape) ** 2
    lam = np.maximum(rho * rng.uniform(3000.0, 6000.0, J.shape) ** 2 - 2 * mu, 0.1 * mu)
    Q = np.ascontiguousarray(random_state(nodes, 31 + order, 1.0, 1.0e6))
    coef = np.ascontiguousarray(np.stack([1.0 / (rho * J), lam / J, mu / J]))
    got = ctypes.c_double()
    assert hostop.host_energy(order, nodes[0], nodes[1], nodes[2], Q.ctypes.data, coef.ctypes.data,
                              ctypes.addressof(got)) == 0
    want = energy(Q, Scheme(order, nodes), J, (rho, lam, mu))
    assert abs(got.value - want) < 1e-12 * want, (got.value, want)


@pytest.mark.parametrize("order,nodes", [(2, (7, 6, 8)), (4, (12, 11, 13)), (6, (16, 17, 18))])
@pytest.mark.parametrize("bcname", sorted(BCS))
def test_traditional_operator_matches_oracle_fp64(hostop, order, nodes, bcname):
    """The traditional operators of Table 2 (OpCoef<kTraditional + order>, D- = D+ = D) through the
    same kernel source, against the oracle's traditional scheme, and its energy."""
    from paper_2011_02600_gb300.opgen import TRADITIONAL
    bc = BCS[bcname]
    X = node_coordinates(make_map("curvy", (1000.0, 1100.0, 900.0)), nodes)
    J, a = metrics(*X, order)
    mat = make_medium("smooth_gradient", Lz=900.0)(*X)
    Q = random_state(nodes, 41 + order, 1.0, 1.0e6)
    sch = Scheme(order, nodes, "traditional")
    got = _host_rhs(hostop, TRADITIONAL + order, Q, J, a, mat, bc)
    want = rhs(Q, sch, J, a, mat, bc)
    err = np.abs(got - want).max(axis=(1, 2, 3)) / np.abs(want).max(axis=(1, 2, 3))
    assert err.max() < 1e-12, err
    rho, lam, mu = mat
    coef = np.ascontiguousarray(np.stack([1.0 / (rho * J), lam / J, mu / J]))
    Qc = np.ascontiguousarray(Q)
    e = ctypes.c_double()
    assert hostop.host_energy(TRADITIONAL + order, *nodes, Qc.ctypes.data, coef.ctypes.data,
                              ctypes.addressof(e)) == 0
    want_e = energy(Q, sch, J, mat)
    assert abs(e.value - want_e) < 1e-12 * want_e


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("geometry", ["curvy", "gaussian_hill"])
def test_kernel_metrics_match_oracle(hostop, order, geometry):
    """The metrics kernel's per-node body (metrics_at: D_c = (D+ + D-)/2 along each axis,
    cofactors by Cramer's rule, Sec. 2.2) gives the oracle's J and a[xi][eta] to rounding; a
    folded mesh is flagged (J <= 0)."""
    nodes = (17, 16, 18)
    ext = (1000.0, 1100.0, 900.0)
    fmap = make_map("curvy", ext) if geometry == "curvy" else \
        make_map("gaussian_hill", ext, hill_amp=300.0, hill_sigma=250.0)
    X = node_coordinates(fmap, nodes)
    xyz = np.ascontiguousarray(np.stack(X))
    jmet = np.zeros((10,) + X[0].shape)
    assert hostop.host_metrics(order, *nodes, xyz.ctypes.data, jmet.ctypes.data) == 0
    J, a = metrics(*X, order)
    assert np.abs(jmet[0] - J).max() < 1e-12 * np.abs(J).max()
    for xi in range(3):
        for c in range(3):
            ref = a[xi][c]
            assert np.abs(jmet[1 + 3 * xi + c] - ref).max() <= 1e-12 * max(np.abs(ref).max(), np.abs(J).max() ** (2 / 3))
    folded = xyz.copy()
    folded[0] = folded[0][:, :, ::-1]          # x reversed along q: J < 0 everywhere
    assert hostop.host_metrics(order, *nodes, folded.ctypes.data, jmet.ctypes.data) == np.prod(nodes)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_source_delta_weights_match_oracle(hostop, order):
    """The 1D discrete-delta weights of sbp_set_sources (source_weights.h: order + 2 nodes,
    moment conditions to degree order + 1; the paper does not describe the discretisation of
    Eq. momententor_pointsource) against the oracle's, at positions across the whole axis
    including both faces and the face-shifted supports; the moment conditions hold directly."""
    from oracle.source import delta_weights_1d
    m = order + 1
    for N in (17, 33, 97):
        h = 1.0 / (N - 1)
        for xi0 in np.concatenate([np.linspace(0.0, 1.0, 257), [h / 3, 1 - h / 3, 0.5 + 1e-12]]):
            start = ctypes.c_int()
            phi = (ctypes.c_double * (m + 1))()
            assert hostop.host_delta_1d(float(xi0), N, m, ctypes.addressof(start), ctypes.addressof(phi)) == 0
            c, want = delta_weights_1d(float(xi0), N, m)
            got = np.array(phi[:])
            assert start.value == c
            assert np.abs(got - want).max() < 1e-9 * max(1.0, np.abs(want).max())
            xs = (np.arange(c, c + m + 1) * h - xi0) / h
            mom = [float(np.sum(got * xs ** k)) for k in range(m + 1)]
            assert abs(mom[0] - 1.0) < 1e-9 and max(abs(v) for v in mom[1:]) < 1e-8 * max(1.0, np.abs(xs).max() ** m)
