"""FGMRES inner solver (FP32 sweeps inside FP64 refinement) and the learned
preconditioner pipeline against the oracle: filter and eigenpairs with the
Jacobi / identity preconditioners, training pairs equal to exact node solves,
and a solve preconditioned by a network trained on such pairs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402

from oracle import feast_nh as OF  # noqa: E402
from oracle.contour import contour_nodes  # noqa: E402
from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402
from paper_1506_04463_gb300 import workloads as wl  # noqa: E402
from gpu_helpers import dev, host, invariants, match_rel  # noqa: E402


@pytest.fixture(scope="module")
def sparse_problem():
    bw = wl.config4(nprob=1, nmin=1200, nmax=1800, seed=5, m0=32)
    A, con = bw.A[0], bw.contours[0]
    n = A.shape[0]
    wk = wl.Workload("random_sparse", A, None, con, 32, bw.Y0[:n], bw.Yh0[:n], "general", bw.exact[0])
    ref = OF.feast_nh(A, None, con, 32, wk.Y0, wk.Yh0, dense=True)
    return wk, ref


@pytest.mark.parametrize("precond", [F.PRECOND_JACOBI, F.PRECOND_NONE])
def test_fgmres_filter_and_solve_match_oracle(sparse_problem, precond):
    wk, ref = sparse_problem
    ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, precision=F.PREC_FP32_IR, inner_kind=F.INNER_FGMRES,
                    precond=precond, krylov_max=600)
    Q, Qh = ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    z, w = contour_nodes(wk.contour)
    Qo, Qho = OF.contour_integration(wk.A, None, OF.node_solvers(wk.A, None, z), z, w, wk.Y0, wk.Yh0)
    assert np.max(np.abs(host(Q) - Qo)) < 1e-9 * np.max(np.abs(Qo))
    assert np.max(np.abs(host(Qh) - Qho)) < 1e-9 * np.max(np.abs(Qho))
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["status"] == F.OK and out["m"] == ref["m"]
    assert match_rel(host(out["lam"]), ref["lam"], 1e-3) < 1e-9
    invariants(wk, out)
    assert out["info"]["krylov_iterations"] > 0 and out["info"]["n_factorizations"] == 0
    ctx.close()


def _convdiff_low(N, beta, m_in=6, m0=16, ne=8):
    A = wl.convdiff2d(N, beta)
    lam = wl.convdiff2d_eigs(N, beta)
    gap = lam[m_in] - lam[m_in - 1]
    c = 0.5 * (lam[0] + lam[m_in - 1])
    a = 0.5 * (lam[m_in - 1] - lam[0]) + 0.5 * gap
    con = wl.Contour(1, complex(c), a, ratio=0.5, angle=0.0, ne=ne)
    n = N * N
    return wl.Workload(f"convdiff{N}", A, None, con, m0, wl.start_block(n, m0, 0), wl.start_block(n, m0, 1),
                       "real", lam[:m_in].astype(np.complex128), {"beta": beta, "N": N})


def test_learned_pairs_are_exact_solves():
    N = 10
    wk = _convdiff_low(N, 15.0)
    ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, precision=F.PREC_FP64)
    rng = np.random.default_rng(2)
    R = rng.standard_normal((N * N, 4)) + 1j * rng.standard_normal((N * N, 4))
    Xin, T = ctx.learned_pairs(dev(R), N, kappa=2.0, features=[0.25])
    Xin_h, T_h = host(Xin), host(T)
    z, _ = contour_nodes(wk.contour)
    ne = len(z)
    for j in range(ne):
        E = OF.NodeSolver(wk.A, None, z[j], dense=True).solve(R)
        for c in range(4):
            s = j * 4 + c
            rms = np.sqrt(np.mean(np.abs(R[:, c]) ** 2))
            e = E[:, c] / rms
            t = T_h[s, ..., 0].ravel() + 1j * T_h[s, ..., 1].ravel()
            assert np.max(np.abs(t - e)) < 1e-5 * np.max(np.abs(e))
            x = Xin_h[s, ..., 0].ravel() + 1j * Xin_h[s, ..., 1].ravel()
            assert np.max(np.abs(x - R[:, c] / rms)) < 1e-6 * np.max(np.abs(R[:, c] / rms))
            assert np.allclose(Xin_h[s, ..., 2], 2.0 * z[j].real, rtol=1e-6)
            assert np.allclose(Xin_h[s, ..., 3], 2.0 * z[j].imag, rtol=1e-6)
            assert np.allclose(Xin_h[s, ..., 4], 0.25) and not Xin_h[s, ..., 5:].any()
    # operator-norm loss: zero output leaves the whole residual (loss = mean |r|^2
    # = 1 for normalised r); the exact correction leaves none
    out = torch.zeros_like(Xin)
    l0, g0 = ctx.operator_loss(out, T, N)
    assert abs(l0 - 1.0) < 1e-5
    out[..., :2] = T
    l1, _ = ctx.operator_loss(out, T, N)
    assert l1 < 1e-9
    # its gradient is 2 M^H y / count with y = M(out - T) = -r at out = 0
    Mh = (np.conj(z[0]) * np.eye(N * N) - wk.A.conj().T.toarray())
    r0 = R[:, 0] / np.sqrt(np.mean(np.abs(R[:, 0]) ** 2))
    gref = 2.0 * (Mh @ (-r0)) / (ne * 4 * N * N)
    g = host(g0)[0, ..., 0].ravel() + 1j * host(g0)[0, ..., 1].ravel()
    assert np.max(np.abs(g - gref)) < 1e-5 * np.max(np.abs(gref))
    ctx.close()


def test_learned_preconditioner_solve_matches_oracle():
    # the learned-preconditioner protocol at 24 x 24: a network trained with the
    # operator-norm loss on exact-solve pairs of 12 operators of the family
    # (Peclet ~ U(1, 50), seeded), then a held-out operator (Peclet 5) solved with
    # FGMRES preconditioned by the network and without a preconditioner.  The
    # FP64 refinement decides the residual, so both give the oracle's eigenpairs;
    # on this operator the network saves FGMRES iterations (on most high-Peclet
    # draws neither form converges, and the network does not help there)
    N, layers = 24, 4
    rng = np.random.default_rng(0)
    net = F.Net(layers, N, 256)
    params = np.concatenate([np.concatenate([rng.standard_normal(9 * 32 * 32) * np.sqrt(2.0 / (9 * 32)) * 0.5,
                                             np.zeros(32)]) for _ in range(layers)]).astype(np.float32)
    net.set_params(params)
    first, last = [], []
    for inst in range(12):
        beta = float(rng.uniform(1, 50))
        wk = _convdiff_low(N, beta)
        kappa = 1.0 / (abs(wk.contour.center) + wk.contour.r)
        ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, precision=F.PREC_FP64)
        R = rng.standard_normal((N * N, 16)) + 1j * rng.standard_normal((N * N, 16))
        Xin, T = ctx.learned_pairs(dev(R), N, kappa=kappa, features=[beta / 50.0])
        losses = F.train_operator_loss(net, ctx, Xin, T, N, steps=150, lr=1e-3, batch=64,
                                       generator=torch.Generator().manual_seed(inst))
        first.append(np.mean(losses[:20]))
        last.append(np.mean(losses[-20:]))
        ctx.close()
    assert np.mean(last) < 0.5 * np.mean(first)
    beta = 5.0
    wk = _convdiff_low(N, beta)
    kappa = 1.0 / (abs(wk.contour.center) + wk.contour.r)
    ref = OF.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=True)
    its = {}
    for name, pc in [("none", F.PRECOND_NONE), ("learned", F.PRECOND_LEARNED)]:
        ctx = F.FeastNH(wk.A, None, wk.contour, wk.m0, precision=F.PREC_FP32_IR, inner_kind=F.INNER_FGMRES,
                        precond=pc, krylov_max=1500, krylov_restart=30, inner_max=4, max_iter=3)
        if pc == F.PRECOND_LEARNED:
            ctx.set_network(net, N, kappa=kappa, features=[beta / 50.0])
        out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
        assert out["status"] == F.OK and out["m"] == ref["m"] == 6
        assert match_rel(host(out["lam"]), ref["lam"], 1e-3) < 1e-9
        invariants(wk, out)
        its[name] = out["info"]["krylov_iterations"]
        ctx.close()
    assert its["learned"] < its["none"], its
    net.close()
