"""Many independent problems in one solve (feast_nh_batch_*) against the FP64
oracle, problem by problem: random sparse nonsymmetric matrices (rows of 9
entries, diagonal shifted by U(0, 4)) of uneven sizes, each with its own
circle at the right edge of its spectrum; the scaled-down members of that
family (n <= 3000) that the oracle solves with dense LU per node."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from oracle import feast_nh as OF  # noqa: E402
from oracle.contour import alpha, contour_nodes, inside  # noqa: E402
from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402
from paper_1506_04463_gb300 import workloads as wl  # noqa: E402
from gpu_helpers import dev, host, match_rel  # noqa: E402


@pytest.fixture(scope="module")
def family():
    bw = wl.config4(nprob=4, nmin=1500, nmax=3000, seed=3)
    refs = []
    for p, A in enumerate(bw.A):
        o, n = bw.offsets[p], A.shape[0]
        refs.append(OF.feast_nh(A, None, bw.contours[p], bw.m0, bw.Y0[o:o + n], bw.Yh0[o:o + n], dense=True))
    return bw, refs


def _check_problem(A, con, out, ref):
    assert out["m"] == ref["m"] >= 16
    lam = host(out["lam"])
    assert match_rel(lam, ref["lam"], 1e-3) < 1e-9
    assert np.all(inside(lam, con))
    X, Xh = host(out["X"]), host(out["Xh"])
    assert np.max(np.abs(Xh.conj().T @ X - np.eye(X.shape[1]))) < 1e-10
    r = OF.residuals(A, None, lam, X, Xh, alpha(con))
    assert np.all(r < 1e-10), r.max()
    assert np.allclose(host(out["res"]), r, rtol=1e-3, atol=1e-14)


@pytest.mark.parametrize("prec", [F.PREC_FP32_IR, F.PREC_FP64])
def test_batch_matches_oracle(family, prec):
    bw, refs = family
    b = F.FeastBatch(bw.A, bw.contours, bw.m0, precision=prec)
    out = b.solve(dev(bw.Y0), dev(bw.Yh0))
    assert out["status"] == F.OK
    inf = out["info"]
    assert inf["converged_problems"] == len(bw.A) and inf["inner_fail"] == 0
    assert inf["threads"] > 0 and inf["tile_rows"] > 0 and inf["grid"] > 0 and inf["krylov_iterations"] > 0
    assert inf["graph"] == 1  # the contour integration replayed as a CUDA graph
    for p, A in enumerate(bw.A):
        _check_problem(A, bw.contours[p], out["problems"][p], refs[p])
        assert abs(out["problems"][p]["iterations"] - refs[p]["iterations"]) <= 2
    # a second solve on the same batch repeats the first exactly
    again = b.solve(dev(bw.Y0), dev(bw.Yh0))
    for p in range(len(bw.A)):
        assert torch.equal(again["problems"][p]["lam"], out["problems"][p]["lam"])
    b.close()


def test_batch_custom_contour_and_single_problem(family):
    # custom nodes/weights (contour kind 2, here the circle's trapezoid rule):
    # the inside test is then the polygon through the nodes, for the library
    # and the oracle alike; a batch of one problem is a valid batch
    bw, _ = family
    p = 1
    z, w = contour_nodes(bw.contours[p])
    con = wl.Contour(2, 0j, 1.0, z=z, w=w)
    o, n = bw.offsets[p], bw.A[p].shape[0]
    ref = OF.feast_nh(bw.A[p], None, con, bw.m0, bw.Y0[o:o + n], bw.Yh0[o:o + n], dense=True)
    b = F.FeastBatch([bw.A[p]], [con], bw.m0, precision=F.PREC_FP32_IR)
    out = b.solve(dev(bw.Y0[o:o + n]), dev(bw.Yh0[o:o + n]))
    assert out["status"] == F.OK
    _check_problem(bw.A[p], con, out["problems"][0], ref)
    b.close()


def test_batch_rejects_bad_arguments(family):
    bw, _ = family
    with pytest.raises(F.FeastError) as e:
        F.FeastBatch(bw.A[:2], [bw.contours[0], wl.Contour(0, 1.0, 0.5, ne=4)], bw.m0)
    assert e.value.status == F.EINVAL
    with pytest.raises(F.FeastError) as e:
        F.FeastBatch(bw.A[:1], bw.contours[:1], bw.m0, inner_kind=F.INNER_BANDED)
    assert e.value.status == F.EINVAL
