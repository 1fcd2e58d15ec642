"""feast_nh_multishift_residual_noalloc against feast_nh_multishift_residual.

The no-allocation entry point serves callers that cannot allocate device
memory (their device memory is owned by their own pool or budget, or their
loop cannot take cudaMalloc's synchronisation).  It must give the same R and
Q as the context-based entry point, and norms that match those of R, on two
calls in a row (its scratch is a shared static device array).  This file is
collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402

from paper_1506_04463_gb300 import build  # noqa: E402
from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402
from paper_1506_04463_gb300 import workloads as wl  # noqa: E402


def _case(with_b):
    n, m, ne = 1237, 24, 8
    A = wl.banded_random(n, 4, 3, 5)
    B = None
    if with_b:
        rng = np.random.default_rng(9)
        B = sp.diags(rng.uniform(1, 2, n) * np.exp(1j * rng.uniform(-0.3, 0.3, n))).tocsr()
    con = wl.Contour(1, 0.2 - 0.1j, 1.5, ratio=0.6, angle=0.4, ne=ne)
    return A, B, con, n, m, ne


@pytest.mark.parametrize("with_b", [False, True])
def test_noalloc_matches_context_entry_point(with_b):
    build.build()
    A, B, con, n, m, ne = _case(with_b)
    ctx = F.FeastNH(A, B, con, m)
    gen = torch.Generator(device="cuda").manual_seed(3)
    for call in range(2):
        X = torch.randn(ne, n, m, dtype=torch.complex128, device="cuda", generator=gen)
        BY = torch.randn(n, m, dtype=torch.complex128, device="cuda", generator=gen)
        R0, Q0 = ctx.multishift_residual(X, BY)
        R1, Q1, rel = F.multishift_residual_noalloc(ctx.A_dev, ctx.B_dev, con, X, BY)
        torch.cuda.synchronize()
        scale_r = R0.abs().max().item()
        assert (R1 - R0).abs().max().item() <= 1e-13 * scale_r, call
        assert (Q1 - Q0).abs().max().item() <= 1e-13 * Q0.abs().max().item(), call
        ref = (R0.abs() ** 2).sum(dim=1).sqrt() / (BY.abs() ** 2).sum(dim=0).sqrt()[None, :]
        assert ((rel - ref).abs() / ref).max().item() < 1e-12, call
    ctx.close()


def test_noalloc_rejects_oversize():
    build.build()
    A, B, con, n, m, ne = _case(False)
    ctx = F.FeastNH(A, None, con, m)
    X = torch.zeros(ne, n, 129, dtype=torch.complex128, device="cuda")
    BY = torch.zeros(n, 129, dtype=torch.complex128, device="cuda")
    with pytest.raises(F.FeastError) as e:
        F.multishift_residual_noalloc(ctx.A_dev, None, con, X, BY)
    assert e.value.status == F.EINVAL
    ctx.close()
