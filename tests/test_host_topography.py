"""The topography-map check of sbp_set_material on the CPU: tests/host_topo.cpp compiles its
per-node body (csrc/topo_check.h) as host C++ and applies it to the oracle's FP64 metrics.  On
the workloads' Gaussian-hill and sinusoidal-topography maps (x = L_x q, y = L_y r) every node is
within rounding of a_q = (a_q,x, 0, 0), a_r = (0, (L_x / L_y) a_q,x, 0); a curvilinear map, a
non-square block's ratio taken wrong, and a single perturbed metric entry are far outside the
library's bound (1e-11)."""
import ctypes

import numpy as np
import pytest

from oracle.metrics import metrics
from workloads.geometry import make_map, node_coordinates

from host_build import build

BOUND = 1e-11


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = build("host_topo.cpp", tmp_path_factory.mktemp("hosttopo") / "libhosttopo.so", shared=True)
    L = ctypes.CDLL(so)
    L.host_topography_deviation.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 3 + [ctypes.c_double]
    L.host_topography_deviation.restype = ctypes.c_double
    return L


def _jmet(name, extent, nodes, order=6):
    X = node_coordinates(make_map(name, extent), nodes)
    J, a = metrics(*X, order)
    f = [J] + [a[xi][eta] for xi in range(3) for eta in range(3)]
    return np.ascontiguousarray(np.stack(f), dtype=np.float64)


def _dev(lib, jm, c=None):
    if c is None:
        c = jm[5].flat[0] / jm[1].flat[0]
    ns, nr, nq = jm.shape[1:]
    return lib.host_topography_deviation(jm.ctypes.data, nq, nr, ns, c)


@pytest.mark.parametrize("name,extent,nodes", [("gaussian_hill", (20000.0, 20000.0, 15000.0), (33, 29, 25)),
                                               ("sinusoids", (60000.0, 60000.0, 24000.0), (41, 37, 21)),
                                               ("gaussian_hill", (30000.0, 20000.0, 15000.0), (35, 27, 19))])
def test_topography_maps_pass(lib, name, extent, nodes):
    jm = _jmet(name, extent, nodes)
    assert _dev(lib, jm) < BOUND
    # the ratio is L_x / L_y (the node spacing of the reference grid cancels)
    assert abs(jm[5].flat[0] / jm[1].flat[0] - extent[0] / extent[1]) < 1e-12 * extent[0] / extent[1]


def test_other_maps_and_planted_departures_fail(lib):
    assert _dev(lib, _jmet("curvy", (1000.0, 1100.0, 900.0), (21, 19, 17))) > 1e-3
    jm = _jmet("gaussian_hill", (30000.0, 20000.0, 15000.0), (35, 27, 19))
    assert _dev(lib, jm, c=1.0) > 0.1                      # the wrong ratio on a non-square block
    jm[2, 7, 11, 13] = 1e-9 * jm[1, 7, 11, 13]              # one node's a_q,y
    assert 1e-10 < _dev(lib, jm) < 1e-8
    jm[2, 7, 11, 13] = np.nan
    assert _dev(lib, jm) == np.inf
