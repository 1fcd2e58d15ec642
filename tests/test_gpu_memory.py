"""Workspace from the library's memory pool: contexts created after others
were destroyed (reusing their memory) and after feast_nh_release_memory give
bit-identical results; a batch and a context alternate on the same pool."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402
from gpu_helpers import dev, host, make_ctx  # noqa: E402
from test_gpu_parity import banded_workload  # noqa: E402


def test_reused_and_released_workspace():
    wk = banded_workload(n=300, kl=4, ku=3, m0=8, ne=8)
    outs = []
    for k in range(4):
        ctx = make_ctx(wk, precision=F.PREC_FP32_IR)
        out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
        outs.append((out["status"], out["m"], host(out["lam"]), host(out["X"])))
        ctx.close()
        if k == 1:
            F.release_memory()
    st0, m0, lam0, X0 = outs[0]
    assert st0 == F.OK and m0 >= 1
    for st, m, lam, X in outs[1:]:
        assert st == st0 and m == m0
        assert np.array_equal(lam, lam0) and np.array_equal(X, X0)
    F.release_memory()
