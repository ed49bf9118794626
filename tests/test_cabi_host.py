"""CPU tests of the C ABI: the library loads, exports every declared symbol, and
rejects invalid arguments on the host (no compute calls, no GPU needed)."""
import os
import re

import pytest

from paper_2011_02600_gb300 import _lib as L
from paper_2011_02600_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "sbp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(sbp_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTED)


def test_min_nodes(lib):
    """2b + max(r, q) for every operator code, against the oracle's own minimum sizes."""
    from oracle.operators import min_nodes, traditional_min_nodes
    assert L.sbp_min_nodes(2) == 6 and L.sbp_min_nodes(4) == 11 and L.sbp_min_nodes(6) == 16
    for order in range(2, 8):
        assert L.sbp_min_nodes(order) == min_nodes(order)
    for order in (2, 4, 6):   # also the bound of the upwind pair that forms the metric terms
        assert L.sbp_min_nodes(L.SBP_TRADITIONAL + order) == max(traditional_min_nodes(order), min_nodes(order))
    for bad in (1, 8, 9, 100, 103, 105, 107):
        with pytest.raises(L.SbpError) as e:
            L.sbp_min_nodes(bad)
        assert e.value.code == 1


def _expect(code, fn, *a):
    with pytest.raises(L.SbpError) as e:
        fn(*a)
    assert e.value.code == code, str(e.value)


def test_create_grid_validation(lib):
    free = [("free",)] * 6
    _expect(1, L.sbp_create_grid, (15, 20, 20), 6, 32, free)        # too few nodes for order 6
    _expect(1, L.sbp_create_grid, (20, 20, 20), 8, 32, free)        # order 8: no closure
    _expect(1, L.sbp_create_grid, (20, 20, 20), 103, 32, free)      # no odd traditional operator
    _expect(1, L.sbp_create_grid, (15, 15, 15), 7, 32, free)        # order 7 needs 16 nodes
    _expect(1, L.sbp_create_grid, (15, 16, 16), 106, 32, free)      # traditional 6 needs 16 (metric terms)
    # the odd upwind orders and the traditional operators (codes 100 + 2, 4, 6) are accepted
    for order in (3, 5, 7, 102, 104, 106):
        L.sbp_destroy(L.sbp_create_grid((20, 20, 20), order, 32, free))
    _expect(1, L.sbp_create_grid, (20, 20, 20), 4, 16, free)        # precision
    _expect(1, L.sbp_create_grid, (20, 20, 20), 4, 32, [("char", 1.5)] + free[1:])
    _expect(1, L.sbp_create_grid, (40000, 40000, 4000), 2, 32, free)  # over 2^31 elements per field
    h = L.sbp_create_grid((33, 17, 16), 6, 32, free)
    ldq, fs, elem = L.sbp_layout(h)
    assert elem == 4 and ldq == 64 and ldq % 32 == 0 and fs % 64 == 0 and fs >= ldq * 17 * 16
    L.sbp_destroy(h)
    h = L.sbp_create_grid((33, 17, 16), 6, 64, free)
    ldq, fs, elem = L.sbp_layout(h)
    assert elem == 8 and ldq == 48 and (fs * 8) % 256 == 0
    L.sbp_destroy(h)


def test_calls_out_of_sequence_are_rejected(lib):
    h = L.sbp_create_grid((16, 16, 16), 6, 32, [("free",)] * 6)
    _expect(5, L.sbp_rhs, h, 256, 512, None)       # before sbp_bind
    _expect(5, L.sbp_step_n, h, 1, 1e-3, None)
    _expect(5, L.sbp_energy, h, None)
    _expect(1, L.sbp_bind, h, 0, 256, 512, 768, 1024)          # null
    _expect(1, L.sbp_bind, h, 256, 256, 512, 768, 1024)        # aliasing
    _expect(1, L.sbp_bind, h, 260, 512, 768, 1024, 1280)       # misaligned
    _expect(1, L.sbp_set_time, h, 0.0, -1)                       # receivers would write before column 0
    _expect(1, L.sbp_set_time, h, float("nan"), 0)
    L.sbp_set_time(h, 2.5, 7)
    assert L.sbp_get_time(h) == (2.5, 7)
    L.sbp_destroy(h)


def test_rk_coefficients_match_published_scheme(lib):
    A, Bc, C = L.sbp_rk_coefficients()
    from oracle import rk
    for k in range(5):
        assert A[k] == rk.A[k] and Bc[k] == rk.B[k]
        assert abs(C[k] - rk.C[k]) < 1e-15


def test_generated_coefficients_match_oracle():
    """The kernel header's closures (package generator) equal the oracle's (independent derivation)."""
    from fractions import Fraction
    from oracle import operators as op
    from paper_2011_02600_gb300 import opgen
    for order in opgen.ORDERS:
        b, r, q, alpha, w, dp, dm = opgen.derive(order)
        H, Dm, Dp, _, _ = op.upwind_pair_exact(order, op.min_nodes(order))
        assert w == H[:b]
        for i in range(b):
            for j in range(b + q):
                assert dp[i][j] == Dp[i][j] and dm[i][j] == Dm[i][j]
        assert alpha == {j: Fraction(a) for j, a in op.interior_stencil(order).items()}
    text = open(os.path.join(ROOT, "paper_2011_02600_gb300", "csrc", "sbp_coeffs.h")).read()
    assert text == opgen.render()


def test_network_entry_points_reject_bad_arguments(lib):
    """The layer kernels' entry points check sizes, leading dimensions and pointers on the host
    (SBP_ERR_ARG) before any launch; fake aligned addresses suffice since nothing runs."""
    a, b, c = 4096, 8192, 16384
    _expect(1, L.sbp_nn_gemm, 0, 8, 8, a, 8, 0, b, 8, 0, c, 8, 0, None, 0, 0.0, None)     # M = 0
    _expect(1, L.sbp_nn_gemm, 8, 8, 8, None, 8, 0, b, 8, 0, c, 8, 0, None, 0, 0.0, None)  # null A
    _expect(1, L.sbp_nn_gemm, 8, 8, 16, a, 8, 0, b, 8, 0, c, 8, 0, None, 0, 0.0, None)   # lda < K
    _expect(1, L.sbp_nn_gemm, 8, 16, 8, a, 8, 0, b, 8, 0, c, 16, 0, None, 0, 0.0, None)  # ldb < N
    _expect(1, L.sbp_nn_gemm, 8, 8, 8, a, 8, 0, b, 8, 0, c, 8, 1, None, 0, 1.0, None)    # beta with BF16 C
    _expect(1, L.sbp_nn_im2col, a, b, 0, 2, 8, 5, 2, None)
    _expect(1, L.sbp_nn_moment_combine, None, None, None, None, None, 4, 2, 8, 0, None)
    _expect(1, L.sbp_nn_moment_combine, a, b, None, None, None, 4, 2, 8, 0, None)        # no output


def test_energy_noalloc_rejects_bad_arguments_on_the_host(lib):
    """Every check of sbp_energy_noalloc runs before its first CUDA call, so it runs without a GPU
    (the addresses below are never dereferenced)."""
    q, mat, nodes = 4096, 8192, (20, 20, 20)
    ldq, fs = 32, 32 * 20 * 20
    _expect(1, L.sbp_energy_noalloc, None, mat, nodes, ldq, fs, 6, 32, 0, None)       # null state
    _expect(1, L.sbp_energy_noalloc, q, mat, nodes, ldq, fs, 5, 32, 0, None)          # order
    _expect(1, L.sbp_energy_noalloc, q, mat, nodes, ldq, fs, 6, 16, 0, None)          # precision
    _expect(1, L.sbp_energy_noalloc, q, mat, (15, 20, 20), ldq, fs, 6, 32, 0, None)   # too few nodes
    _expect(1, L.sbp_energy_noalloc, q, mat, nodes, 19, fs, 6, 32, 0, None)           # ldq < nq
    _expect(1, L.sbp_energy_noalloc, q, mat, nodes, ldq, fs - 1, 6, 32, 0, None)      # fields overlap
    _expect(1, L.sbp_energy_noalloc, q, mat, nodes, ldq, 1 << 31, 6, 32, 0, None)     # field stride >= 2^31
    _expect(1, L.sbp_energy_noalloc, q, mat, nodes, ldq, fs, 6, 32, 4097, None)       # beyond the static scratch
    _expect(1, L.sbp_energy_noalloc, q, mat, nodes, ldq, fs, 6, 32, -1, None)


def test_generated_traditional_coefficients_match_oracle():
    """The kernel header's traditional operators (OpCoef<kTraditional + order>, package generator)
    equal the oracle's (independent derivation): norm, and both closure tables equal to D."""
    from oracle import operators as op
    from paper_2011_02600_gb300 import opgen
    for order in (2, 4, 6):
        b, r, q, alpha, w, dp, dm = opgen.derive(opgen.TRADITIONAL + order)
        N = op.traditional_min_nodes(order) + 3
        H, D, _, _ = op.traditional_exact(order, N)
        assert w == H[:b] and dp == dm
        for i in range(b):
            for j in range(len(dp[i])):
                assert dp[i][j] == D[i][j]
        assert alpha == op.traditional_stencil(order)


def test_set_slab_validation(lib):
    """sbp_set_slab (an s-slab of a decomposed block): ghost counts of 0 exactly at the block's
    faces and at least the stencil's reach elsewhere, planes inside the block, a face slab big
    enough for its closures, and only before sbp_bind."""
    free = [("free",)] * 6
    h = L.sbp_create_grid((20, 20, 24), 4, 64, free)
    for bad in [(60, 10, 2, 3), (60, 0, 3, 3), (60, 40, 3, 0), (60, 50, 3, 3), (8, 0, 0, 3), (60, 10, 3, 3 - 3),
                (24, 0, 0, 0 + 1)]:
        _expect(1, L.sbp_set_slab, h, *bad)
    L.sbp_set_slab(h, 60, 10, 3, 3)       # interior slab: planes 10..33 of 60
    L.sbp_set_slab(h, 60, 0, 0, 3)        # low face slab
    L.sbp_set_slab(h, 60, 36, 3, 0)       # high face slab
    L.sbp_set_slab(h, 24, 0, 0, 0)        # the whole block again
    L.sbp_destroy(h)


def test_interface_face_validation(lib):
    """Interface faces (SBP_BC_INTERFACE): accepted by sbp_create_grid; sbp_set_interface only on
    such a face and a face index in 0..5; the interface trace needs a bound grid with material."""
    bc = [("free",), ("interface",), ("free",), ("free",), ("free",), ("char", 0.0)]
    h = L.sbp_create_grid((20, 20, 20), 4, 32, bc)
    L.sbp_set_interface(h, 1, None)
    _expect(1, L.sbp_set_interface, h, 0, None)       # not an interface face
    _expect(1, L.sbp_set_interface, h, 6, None)
    _expect(5, L.sbp_interface_trace, h, 1, None, 0x1000, None)   # not bound
    L.sbp_destroy(h)


def test_map_path_and_adjoint_step_checks_on_the_host(lib):
    """The metric-path calls and the whole-step adjoint validate on the host: an unknown path is
    refused, an unbound grid reports the general path and refuses the adjoint step, and the
    Fourier-feature entry point checks its sizes before any launch."""
    h = L.sbp_create_grid((20, 20, 20), 4, 32, [("free",)] * 6)
    assert L.sbp_map_path(h) == L.SBP_MAP_GENERAL          # no material yet
    _expect(1, L.sbp_set_map_path, h, 2)                    # TOPOGRAPHY is reported, not requested
    _expect(1, L.sbp_set_map_path, h, -1)
    L.sbp_set_map_path(h, L.SBP_MAP_GENERAL)
    L.sbp_set_map_path(h, L.SBP_MAP_AUTO)
    _expect(5, L.sbp_adjoint_step, h, 1e-3, 4096, 8192, 16384, 32768, 65536, 131072, None)   # before sbp_bind
    L.sbp_destroy(h)
    _expect(1, L.sbp_nn_fourier_features, None, 4096, 3, 8, 4, None)     # null input
    _expect(1, L.sbp_nn_fourier_features, 4096, 8192, 0, 8, 4, None)     # no inputs
    _expect(1, L.sbp_nn_fourier_features, 4096, 8192, 3, 8, 17, None)    # too many frequencies
