"""Host-side checks of the C ABI: the library loads, exports every declared
entry point, and its host-only functions agree with the oracle (no GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle.contour import contour_nodes
from paper_1506_04463_gb300 import feast_nh as F
from paper_1506_04463_gb300.workloads import Contour

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1506_04463_gb300 import build
    build.build()
    return F.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "feast_nh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(feast_nh_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    assert sorted(F.EXPORTS) == names


def test_default_opts_and_strerror(L):
    o = F.default_opts()
    assert (o.eps, o.eta, o.mu, o.inner_tol, o.max_iter) == (1e-10, 1e-16, 0.1, 1e-10, 100)
    for s in range(8):
        assert len(L.feast_nh_strerror(s)) > 3


@pytest.mark.parametrize("con", [Contour(0, 2.0 + 0.5j, 0.3, ne=8), Contour(1, 1 + 1j, 2.0, 0.5, 0.3, ne=16),
                                 Contour(1, 0.0588, 0.0019, 0.5, 0.0, ne=16)])
def test_library_nodes_match_oracle(L, con):
    z, w = F.nodes(con)
    zo, wo = contour_nodes(con)
    assert np.max(np.abs(z - zo)) < 1e-15 * (1 + abs(con.center))
    assert np.max(np.abs(w - wo)) < 1e-16 * (1 + con.r)


def test_custom_nodes_roundtrip(L):
    zo = np.exp(2j * np.pi * np.arange(5) / 5)
    wo = zo / 5
    z, w = F.nodes(Contour(2, 0j, 1.0, z=zo, w=wo))
    assert np.array_equal(z, zo) and np.array_equal(w, wo)


def test_init_rejects_bad_arguments_without_gpu(L):
    h = C.c_void_p()
    con, _ = F.contour_struct(Contour(0, 0j, 1.0, ne=8))
    o = F.default_opts()
    # NULL matrix
    assert L.feast_nh_init(C.byref(h), None, None, C.byref(con), 4, C.byref(o), None) == F.EINVAL
    # bad m0 / ne are rejected before any device work
    a = F.Csr(10, 10, 8, 8, 8, F.R64)  # dummy non-null pointers, never dereferenced
    assert L.feast_nh_init(C.byref(h), C.byref(a), None, C.byref(con), 0, C.byref(o), None) == F.EINVAL
    assert L.feast_nh_init(C.byref(h), C.byref(a), None, C.byref(con), 129, C.byref(o), None) == F.EINVAL
    con.ne = 0
    assert L.feast_nh_init(C.byref(h), C.byref(a), None, C.byref(con), 4, C.byref(o), None) == F.EINVAL
    assert h.value is None
    assert L.feast_nh_nodes(None, None, None) == F.EINVAL


def test_shifted_residual_definition():
    # oracle helper used by the GPU parity test of the multi-shift product
    from oracle.feast_nh import shifted_residuals
    import scipy.sparse as sp
    A = sp.diags([1.0, 2.0, 3.0]).tocsr()
    X = np.ones((2, 3, 1), complex)
    R, Q = shifted_residuals(A, None, np.array([1j, 2.0]), np.array([0.5, 0.25]), X, np.zeros((3, 1)))
    assert np.allclose(R[0, :, 0], -(1j - np.array([1, 2, 3])))
    assert np.allclose(Q, 0.75)


def test_new_entry_points_reject_null_context(L):
    assert L.feast_nh_small_eig(None, None, 4, None, None) == F.EINVAL
    assert L.feast_nh_inject_device_error(None, F.DEVERR_TIMEOUT) == F.EINVAL
    assert L.feast_nh_multishift_residual(None, None, None, None, None, 4, 0) == F.EINVAL
