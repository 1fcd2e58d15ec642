"""feast_nh_multishift_residual_noalloc against feast_nh_multishift_residual.

The no-allocation entry point serves callers that cannot allocate device
memory: their device memory is owned by their own pool or budget, or their
loop cannot take the synchronisation of cudaMalloc/cudaFree.  It must give the
same R and Q as the context-based entry point, and norms that match those of
R, on two calls in a row (its scratch is one shared static device array that
keeps the last call's contents), for every contour kind, with and without Q,
and for a small call that follows a larger one (fewer partial-sum CTAs,
smaller m: no stale scratch may be read).  This file is collected last on
purpose."""
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


def _contour(kind, ne):
    if kind == 0:
        return wl.Contour(0, 0.3 + 0.2j, 1.2, ne=ne)
    if kind == 1:
        return wl.Contour(1, 0.2 - 0.1j, 1.5, ratio=0.6, angle=0.4, ne=ne)
    t = 2 * np.pi * (np.arange(ne) + 0.25) / ne
    z = 0.1 + 1.3 * np.cos(t) + 0.9j * np.sin(t)
    w = (-1.3 * np.sin(t) + 0.9j * np.cos(t)) / (1j * ne)
    return wl.Contour(2, 0j, 1.0, z=z, w=w)


def _case(n, m, ne, kind, with_b, seed):
    A = wl.banded_random(n, 4, 3, seed)
    B = None
    if with_b:
        rng = np.random.default_rng(seed + 9)
        B = sp.diags(rng.uniform(1, 2, n) * np.exp(1j * rng.uniform(-0.3, 0.3, n))).tocsr()
    return A, B, _contour(kind, ne)


def _check_pair(ctx, con, X, BY, want_q):
    R0, Q0 = ctx.multishift_residual(X, BY)
    R1, Q1, rel = F.multishift_residual_noalloc(ctx.A_dev, ctx.B_dev, con, X, BY, want_q=want_q)
    torch.cuda.synchronize()
    assert (R1 - R0).abs().max().item() <= 1e-13 * R0.abs().max().item()
    if want_q:
        assert (Q1 - Q0).abs().max().item() <= 1e-13 * Q0.abs().max().item()
    else:
        assert Q1 is None
    ref = (R0.abs() ** 2).sum(dim=1).sqrt() / (BY.abs() ** 2).sum(dim=0).sqrt()[None, :]
    assert ((rel - ref).abs() / ref).max().item() < 1e-12


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("with_b,want_q", [(False, True), (True, True), (True, False)])
def test_noalloc_matches_context_entry_point(kind, with_b, want_q):
    build.build()
    n, m, ne = 1237, 24, 8
    A, B, con = _case(n, m, ne, kind, with_b, 5)
    ctx = F.FeastNH(A, B, con, m)
    gen = torch.Generator(device="cuda").manual_seed(3)
    for call in range(2):
        X = torch.randn(ne, n, m, dtype=torch.complex128, device="cuda", generator=gen)
        BY = torch.randn(n, m, dtype=torch.complex128, device="cuda", generator=gen)
        _check_pair(ctx, con, X, BY, want_q)
    ctx.close()


def test_noalloc_small_call_after_large_call():
    # a large call (many partial-sum CTAs, m = 64) leaves its partials in the
    # shared scratch; the small call after it (n = 300, m = 8) must not read them
    build.build()
    gen = torch.Generator(device="cuda").manual_seed(7)
    for (n, m, ne, kind) in [(60000, 64, 16, 1), (300, 8, 4, 0)]:
        A, B, con = _case(n, m, ne, kind, True, n)
        ctx = F.FeastNH(A, B, con, m)
        X = torch.randn(ne, n, m, dtype=torch.complex128, device="cuda", generator=gen)
        BY = torch.randn(n, m, dtype=torch.complex128, device="cuda", generator=gen)
        _check_pair(ctx, con, X, BY, True)
        ctx.close()


def test_noalloc_rejects_oversize():
    build.build()
    A, B, con = _case(1237, 24, 8, 1, False, 5)
    ctx = F.FeastNH(A, None, con, 24)
    X = torch.zeros(8, 1237, 129, dtype=torch.complex128, device="cuda")
    BY = torch.zeros(1237, 129, dtype=torch.complex128, device="cuda")
    with pytest.raises(F.FeastError) as e:
        F.multishift_residual_noalloc(ctx.A_dev, None, con, X, BY)
    assert e.value.status == F.EINVAL
    with pytest.raises(ValueError):
        F.multishift_residual_noalloc(ctx.A_dev, None, con, X[:, :100, :24].contiguous(), BY[:100, :24].contiguous())
    with pytest.raises(TypeError):
        F.multishift_residual_noalloc(ctx.A_dev, None, con, X[:, :, :24].to(torch.complex64), BY[:, :24])
    ctx.close()
