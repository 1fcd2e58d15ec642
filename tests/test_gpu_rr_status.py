"""CUDA path against the oracle on the parts of the method that the end-to-end
tests reach only indirectly: the resize of eq. (resize), the per-iteration
counts m_tilde, m_r, m_s of steps 3.b, 5.a and the spurious test of Sec. 2.7,
m0 = 128, the small dense eigensolver against LAPACK, the single-precision
residual output, and the status codes of inner-solve failure and of the
device error word (fault injected on the host)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import scipy.linalg as sla  # noqa: E402

from oracle import feast_nh as OF  # noqa: E402
from oracle.contour import contour_nodes  # noqa: E402
from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402
from paper_1506_04463_gb300 import workloads as wl  # noqa: E402
from gpu_helpers import dev, host, invariants, make_ctx, match_rel  # noqa: E402
from test_gpu_parity import banded_workload  # noqa: E402


def _stepwise(ctx, Y0, Yh0, max_it):
    """filter + rr through the C ABI, one outer iteration per call pair."""
    Y, Yh = dev(Y0), dev(Yh0)
    hist = []
    for _ in range(max_it):
        Q, Qh = ctx.filter(Y, Yh)
        lam, Y, Yh, info = ctx.rr(Q, Qh)
        hist.append(info)
        if info["converged"]:
            break
    return hist, lam


@pytest.mark.parametrize("prec", [F.PREC_FP64, F.PREC_FP32_IR])
def test_resize_on_rank_deficient_start(prec):
    # eq. (resize): duplicate start columns make B_Q singular; m_tilde = m0 - 1
    wk = wl.pencil_workload(40, 5, ne=8, m0=10)
    Y0, Yh0 = wk.Y0.copy(), wk.Yh0.copy()
    Y0[:, 9] = Y0[:, 8]
    Yh0[:, 9] = Yh0[:, 8]
    oo = OF.feast_nh(wk.A, wk.B, wk.contour, 10, Y0, Yh0, record=True)
    assert oo["history"][0]["m_tilde"] == 9
    ctx = make_ctx(wk, precision=prec)
    hist, _ = _stepwise(ctx, Y0, Yh0, 1)
    assert hist[0]["m_tilde"] == 9
    out = ctx.solve(dev(Y0), dev(Yh0))
    assert out["status"] == F.OK and out["m"] == oo["m"] == wk.exact.size
    assert match_rel(host(out["lam"]), oo["lam"], 1e-3) < 1e-9
    invariants(wk, out)
    ctx.close()


def test_history_matches_oracle():
    # per-iteration m_tilde, m_r, m_s (Sec. 2.7 spurious count) and the
    # iteration of convergence, step by step through feast_nh_filter/_rr
    wk = wl.config2(N=20, m0=48, ne=16)
    oo = OF.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=True, record=True)
    ctx = make_ctx(wk, precision=F.PREC_FP64)
    hist, lam = _stepwise(ctx, wk.Y0, wk.Yh0, len(oo["history"]) + 2)
    assert len(hist) == len(oo["history"])
    for g, o in zip(hist, oo["history"]):
        assert (g["m_tilde"], g["m_r"], g["m_s"]) == (o["m_tilde"], o["m_r"], o["m_s"]), (g, o)
    assert hist[-1]["converged"] and hist[-1]["m_r"] - hist[-1]["m_s"] == 30
    assert hist[0]["m_s"] == 0
    ctx.close()


def test_m0_128():
    # the largest subspace the library accepts (ne * m0 = 2048)
    wk = wl.config2(N=20, m0=128, ne=16)
    oo = OF.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=True)
    for prec in (F.PREC_FP64, F.PREC_FP32_IR):
        ctx = make_ctx(wk, precision=prec)
        out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
        assert out["status"] == F.OK and out["m"] == oo["m"] == 30
        assert match_rel(host(out["lam"]), oo["lam"], 1e-3) < 1e-9
        assert match_rel(host(out["lam"]), wk.exact, 1e-3) < 1e-9
        invariants(wk, out)
        ctx.close()


@pytest.mark.parametrize("m", [8, 33, 64, 128])
def test_small_eig_against_lapack(m):
    rng = np.random.default_rng(100 + m)
    M = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    wk = wl.pencil_workload(40, 3, ne=8, m0=8)
    ctx = make_ctx(wk)
    lam, V = ctx.small_eig(dev(M))
    lam, V = host(lam), host(V)
    ref = sla.eigvals(M)
    nrm = np.linalg.norm(M, 2)
    assert match_rel(lam, ref, nrm) < 1e-12
    # right eigenvectors: M V = V Lambda, columns of unit scale
    assert np.all(np.linalg.norm(V, axis=0) > 0)
    Vn = V / np.linalg.norm(V, axis=0)
    assert np.max(np.abs(M @ Vn - Vn * lam[None, :])) < 1e-12 * nrm
    ctx.close()


def test_multishift_residual_single_precision_output():
    # the refinement residual stored in complex64: the FP64 definition rounded once
    wk = banded_workload(n=257, kl=4, ku=2, m0=7, ne=5)
    ctx = make_ctx(wk, precision=F.PREC_FP32_IR)
    z, w = contour_nodes(wk.contour)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((5, 257, 7)) + 1j * rng.standard_normal((5, 257, 7))
    BY = rng.standard_normal((257, 7)) + 1j * rng.standard_normal((257, 7))
    R, Q = ctx.multishift_residual(dev(X), dev(BY), r_single=True)
    assert R.dtype == torch.complex64
    Ro, Qo = OF.shifted_residuals(wk.A, wk.B, z, w, X, BY)
    Rg = host(R).astype(np.complex128)
    # one rounding to single precision per component
    assert np.all(np.abs(Rg.real - Ro.real) <= 2 ** -23 * np.abs(Ro.real) + 1e-12 * np.max(np.abs(Ro)))
    assert np.all(np.abs(Rg.imag - Ro.imag) <= 2 ** -23 * np.abs(Ro.imag) + 1e-12 * np.max(np.abs(Ro)))
    assert np.max(np.abs(host(Q) - Qo)) < 1e-13 * np.max(np.abs(Qo))
    ctx.close()


@pytest.mark.parametrize("with_b,side,m", [(False, 0, 10), (True, 0, 10), (True, 1, 10), (False, 1, 9)])
def test_multishift_spmm_single_precision(with_b, side, m):
    # the FP32 Krylov operator against the definition (z_j B - A) P_j in FP64
    # (m even: two columns per 16-byte lane load; m odd: one per lane)
    wk = banded_workload(n=331, kl=6, ku=3, m0=10, ne=6, with_b=with_b)
    ctx = make_ctx(wk, precision=F.PREC_FP32_IR)
    z, w = contour_nodes(wk.contour)
    rng = np.random.default_rng(5)
    P = (rng.standard_normal((6, 331, m)) + 1j * rng.standard_normal((6, 331, m))).astype(np.complex64)
    V = host(ctx.multishift_spmm(torch.from_numpy(P).cuda(), side=side)).astype(np.complex128)
    A = wk.A if side == 0 else wk.A.conj().T.tocsr()
    B = None if wk.B is None else (wk.B if side == 0 else wk.B.conj().T.tocsr())
    zz = z if side == 0 else np.conj(z)
    Ro, _ = OF.shifted_residuals(A, B, zz, w, P.astype(np.complex128), np.zeros((331, m)))
    Vo = -Ro
    # single-precision products and sums over at most 11 terms per entry
    absA = abs(A)
    bound = np.stack([(np.abs(zz[j]) * (np.abs(P[j]) if B is None else abs(B) @ np.abs(P[j])) + absA @ np.abs(P[j]))
                      for j in range(6)])
    assert np.all(np.abs(V - Vo) <= 24 * 2 ** -24 * bound + 1e-30)
    ctx.close()


@pytest.mark.parametrize("prec,opts", [(F.PREC_FP32_IR, dict(inner_max=1, inner_tol=1e-14)),
                                       (F.PREC_FP64, dict(inner_tol=1e-30))])
def test_inner_solve_failure_is_reported(prec, opts):
    # a refinement cap (or an unreachable tolerance) that the shifted solves do
    # not meet is a status, not a silent result
    wk = banded_workload(n=300, kl=5, ku=3)
    ctx = make_ctx(wk, precision=prec, **opts)
    with pytest.raises(F.FeastError) as e:
        ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    assert e.value.status == F.EINNER
    ctx.close()
    # the whole solve with single-precision solves only: no convergence, and the
    # status names the inner solves; info counts the filters that missed
    if prec == F.PREC_FP32_IR:
        ctx = make_ctx(wk, precision=prec, max_iter=3, **opts)
        out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
        assert out["status"] == F.EINNER and out["info"]["inner_fail"] >= 1
        ctx.close()


def test_pivot_statistics_reported():
    wk = banded_workload(n=300, kl=5, ku=3)
    ctx = make_ctx(wk, precision=F.PREC_FP32_IR)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    inf = out["info"]
    assert 0 < inf["pivot_min"] <= inf["pivot_max"] < np.inf
    assert inf["inner_fail"] == 0
    ctx.close()


@pytest.mark.parametrize("bits,status", [(F.DEVERR_TIMEOUT, F.ETIMEOUT), (F.DEVERR_ZERO_PIVOT, F.ESINGULAR),
                                         (F.DEVERR_QR_NOCONV, F.ECUDA)])
def test_injected_device_error_maps_to_status(bits, status):
    # the device error word set on the host side (no kernel waits or faults):
    # the call reports the status, and the context stays usable afterwards
    wk = banded_workload(n=300, kl=5, ku=3)
    ctx = make_ctx(wk, precision=F.PREC_FP32_IR)
    ref = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    ctx.inject_device_error(bits)
    with pytest.raises(F.FeastError) as e:
        ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    assert e.value.status == status
    ctx.inject_device_error(bits)
    with pytest.raises(F.FeastError) as e:
        ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert e.value.status == status
    again = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert again["status"] == F.OK and torch.equal(again["lam"], ref["lam"])
    ctx.close()


@pytest.mark.parametrize("defect", ["column", "rowptr"])
def test_malformed_csr_rejected(defect):
    # column indices and row pointers are validated before any kernel
    # scatters through them: a bad CSR is EINVAL, not a fault
    wk = banded_workload(n=120, kl=2, ku=2, m0=6, ne=4, with_b=False)
    rp, ci, val, dt, n, nnz = F.csr_to_device(wk.A)
    if defect == "column":
        ci = ci.clone()
        ci[17] = n                      # one index past the last column
    else:
        rp = rp.clone()
        rp[40] = rp[42] + 1             # row pointers decrease
    with pytest.raises(F.FeastError) as e:
        F.FeastNH((rp, ci, val, dt, n, nnz), None, wk.contour, 6)
    assert e.value.status == F.EINVAL
