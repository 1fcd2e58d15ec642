"""Full-size workload (2D convection-diffusion on 300 x 300, n = 90 000) in the
configuration bench.py times: closed-form spectrum, invariants, and sampled
filter columns against the oracle."""
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
def wk():
    return wl.config2(N=300)


@pytest.mark.parametrize("prec", [F.PREC_FP32_IR, F.PREC_FP64])
def test_fullsize_solve(wk, prec):
    ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, precision=prec)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["status"] == F.OK and out["m"] == 30
    lam = host(out["lam"])
    assert match_rel(lam, wk.exact, 1e-3) < 1e-9
    assert np.all(inside(lam, wk.contour))
    X, Xh = out["X"], out["Xh"]
    G = (Xh.conj().T @ X).cpu().numpy()
    assert np.max(np.abs(G - np.eye(30))) < 1e-10
    r = OF.residuals(wk.A, None, lam, host(X), host(Xh), alpha(wk.contour))
    assert np.all(r < 1e-10)
    ctx.close()


def test_fullsize_filter_sampled_columns(wk):
    # the filter in the bench's launch configuration (all 64 columns, every
    # node, both sides): a 16-column block of Q and Q^ against the oracle
    # (SuperLU per node); columns of the filter are independent systems
    ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, precision=F.PREC_FP32_IR)
    Q, Qh = ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    cols = np.arange(3, 64, 4)[:16]
    Y, Yh = wk.Y0[:, cols].copy(), wk.Yh0[:, cols].copy()
    z, w = contour_nodes(wk.contour)
    Qo, Qho = OF.contour_integration(wk.A, None, OF.node_solvers(wk.A, None, z, dense=False), z, w, Y, Yh)
    Qg, Qhg = host(Q)[:, cols], host(Qh)[:, cols]
    for k in range(cols.size):
        assert np.max(np.abs(Qg[:, k] - Qo[:, k])) < 1e-9 * np.max(np.abs(Qo[:, k])), k
        assert np.max(np.abs(Qhg[:, k] - Qho[:, k])) < 1e-9 * np.max(np.abs(Qho[:, k])), k
    ctx.close()
