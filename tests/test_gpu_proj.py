"""The n x m^2 products of the Rayleigh-Ritz step (B_Q, A_U, B_U of steps 2.a
and 4.a of Fig. alg:three, the block updates of eq. uu and step 4.d) on the
tensor cores, in exact integer-digit products, against FP64 references:

* integer-valued data, whose products and sums FP64 holds exactly: the
  tensor-core result equals the exact result bit for bit;
* random data at ragged sizes (n not a multiple of the 16-row stage, column
  counts not multiples of the 64-column tile, one row, 128 columns): within
  the error bound of the digit truncation, n 2^-51 max|x| max|y| per entry,
  and within the FP64 kernels' own error;
* columns whose scales span 10^-150 .. 10^150 and an all-zero column: the
  per-column power-of-two scaling keeps every entry's relative accuracy;
* the Gram products do not depend on the order of summation (row
  permutations give bit-identical results);
* full solves with either method give the same Ritz pairs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402
from paper_1506_04463_gb300 import workloads as wl  # noqa: E402
from gpu_helpers import dev, host, invariants, make_ctx, match_rel  # noqa: E402
from test_gpu_parity import banded_workload  # noqa: E402


def _ctx(n):
    """A context of size n (the products only use its size and workspace)."""
    A = wl.tridiag_toeplitz(n, 1.0, 2.0, 0.5)
    return F.FeastNH(A, None, wl.Contour(kind=0, center=2.0 + 0j, r=0.08, ne=4), min(8, n))


def _cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _ints(rng, lim, *shape):
    return (rng.integers(-lim, lim + 1, shape) + 1j * rng.integers(-lim, lim + 1, shape)).astype(np.complex128)


@pytest.mark.parametrize("n,mx,my", [(4103, 64, 64), (1000, 37, 100), (777, 128, 128)])
def test_gram_exact_on_integers(n, mx, my):
    # |entries| <= 2^19, n < 2^13: every partial sum is an integer below 2^53,
    # so X^H Y is exact in FP64 and the digit products must reproduce it
    rng = np.random.default_rng(n + mx)
    X, Y = _ints(rng, 2**19, n, mx), _ints(rng, 2**19, n, my)
    ctx = _ctx(n)
    G = host(ctx.gram(dev(X), dev(Y), F.PROJ_TENSOR))
    assert np.array_equal(G, X.conj().T @ Y)
    ctx.close()


@pytest.mark.parametrize("n,mx,my", [(4103, 64, 64), (1000, 37, 100), (2049, 128, 128), (2, 3, 2), (17, 64, 1),
                                     (90001, 64, 64)])
def test_gram_tensor_accuracy(n, mx, my):
    rng = np.random.default_rng(7 * n + my)
    X, Y = _cplx(rng, n, mx), _cplx(rng, n, my)
    ctx = _ctx(n)
    Gt = host(ctx.gram(dev(X), dev(Y), F.PROJ_TENSOR))
    Gf = host(ctx.gram(dev(X), dev(Y), F.PROJ_FP64))
    ref = X.conj().T @ Y
    # digit truncation: <= 2^-51 max|x_a| max|y_b| per term, n terms
    bound = n * 2.0**-51 * np.abs(X).max(0)[:, None] * np.abs(Y).max(0)[None, :]
    fp64 = 4 * n * 2.0**-53 * (np.abs(X).T @ np.abs(Y))  # FP64 dot-product bound
    assert np.all(np.abs(Gt - ref) <= bound + fp64)
    assert np.all(np.abs(Gf - ref) <= fp64)
    assert np.linalg.norm(Gt - ref) <= 1e-14 * np.linalg.norm(ref)
    ctx.close()


def test_gram_independent_of_summation_order():
    # the digit products are summed exactly (integers) and rounded once, so
    # permuting the rows of X and Y together (which moves them between the
    # CTAs' row chunks) leaves G bit-identical; an FP summation would not
    n, m = 50021, 64
    rng = np.random.default_rng(5)
    X, Y = _cplx(rng, n, m), _cplx(rng, n, m)
    perm = rng.permutation(n)
    ctx = _ctx(n)
    G1 = host(ctx.gram(dev(X), dev(Y), F.PROJ_TENSOR))
    G2 = host(ctx.gram(dev(X[perm]), dev(Y[perm]), F.PROJ_TENSOR))
    assert np.array_equal(G1, G2)
    ctx.close()


def test_gram_wide_exponent_range_and_zero_column():
    n, m = 3001, 40
    rng = np.random.default_rng(11)
    sx = 10.0 ** rng.uniform(-150, 150, m)
    sy = 10.0 ** rng.uniform(-150, 150, m)
    X, Y = _cplx(rng, n, m) * sx, _cplx(rng, n, m) * sy
    X[:, 5] = 0
    Y[:, 9] = 0
    ctx = _ctx(n)
    G = host(ctx.gram(dev(X), dev(Y), F.PROJ_TENSOR))
    ref = X.conj().T @ Y
    scale = np.linalg.norm(X, axis=0)[:, None] * np.linalg.norm(Y, axis=0)[None, :]
    assert np.all(G[5, :] == 0) and np.all(G[:, 9] == 0)
    nz = scale > 0
    assert np.max(np.abs(G - ref)[nz] / scale[nz]) < 1e-14
    ctx.close()


@pytest.mark.parametrize("n,mx,mz", [(4103, 64, 64), (1000, 100, 33), (129, 128, 128), (2, 7, 5)])
def test_block_product_exact_on_integers(n, mx, mz):
    rng = np.random.default_rng(n + mz)
    X, S = _ints(rng, 2**20, n, mx), _ints(rng, 2**10, mx, mz)
    ctx = _ctx(n)
    Z = host(ctx.block_product(dev(X), dev(S), F.PROJ_TENSOR))
    assert np.array_equal(Z, X @ S)
    ctx.close()


@pytest.mark.parametrize("n,mx,mz", [(4103, 64, 64), (1000, 100, 33), (2049, 128, 128), (90001, 64, 64)])
def test_block_product_tensor_accuracy(n, mx, mz):
    rng = np.random.default_rng(3 * n + mx)
    X, S = _cplx(rng, n, mx), _cplx(rng, mx, mz)
    # rows of very different scales: the scaling is per row of X
    X *= (10.0 ** rng.uniform(-100, 100, n))[:, None]
    ctx = _ctx(n)
    Zt = host(ctx.block_product(dev(X), dev(S), F.PROJ_TENSOR))
    Zf = host(ctx.block_product(dev(X), dev(S), F.PROJ_FP64))
    ref = X @ S
    bound = mx * 2.0**-51 * np.abs(X).max(1)[:, None] * np.abs(S).max(0)[None, :]
    fp64 = 4 * mx * 2.0**-53 * (np.abs(X) @ np.abs(S))
    assert np.all(np.abs(Zt - ref) <= bound + fp64)
    assert np.all(np.abs(Zf - ref) <= fp64)
    ctx.close()


@pytest.mark.parametrize("prec", [F.PREC_FP64, F.PREC_FP32_IR])
def test_solve_same_with_either_projection(prec):
    wk = banded_workload(n=600, kl=4, ku=3, m0=16, ne=8)
    out = {}
    for proj in (F.PROJ_TENSOR, F.PROJ_FP64):
        ctx = make_ctx(wk, precision=prec, projection=proj)
        out[proj] = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
        assert out[proj]["status"] == F.OK
        invariants(wk, out[proj])
        ctx.close()
    a, b = out[F.PROJ_TENSOR], out[F.PROJ_FP64]
    assert a["m"] == b["m"] >= 1
    assert a["info"]["iterations"] == b["info"]["iterations"]
    la, lb = host(a["lam"]), host(b["lam"])
    assert match_rel(la, lb, np.max(np.abs(lb))) < 1e-12
