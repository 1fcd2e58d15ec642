"""Pins of the oracle's Rayleigh-Ritz, residual and outer loop (Fig. alg:three)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import feast_nh as F
from oracle.contour import alpha, contour_nodes, inside, rho_a
from paper_1506_04463_gb300 import workloads as wl


def _match(a, b):
    """Max relative distance after optimal one-to-one matching."""
    from scipy.optimize import linear_sum_assignment
    a, b = np.asarray(a), np.asarray(b)
    assert a.size == b.size
    C = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(C)
    return np.max(C[r, c] / np.maximum(np.abs(b[c]), 1e-3))


def _invariants(wk, out, tol=1e-10):
    B = wk.B
    X, Xh = out["X"], out["Xh"]
    BX = X if B is None else B @ X
    assert np.max(np.abs(Xh.conj().T @ BX - np.eye(X.shape[1]))) < tol      # X^^H B X = I
    assert np.all(inside(out["lam"], wk.contour))                            # only lambda in C
    assert np.all(out["res"] < 1e-10)


def test_residual_closed_form():
    # A = diag(1, 2), x = [1, t], lambda = 1: ||Ax - x||_1 = |t|, ||alpha x||_1 = alpha (1+|t|).
    A = sp.diags([1.0, 2.0]).tocsr().astype(complex)
    t = 1e-3
    X = np.array([[1.0], [t]], complex)
    r = F.residuals(A, None, np.array([1.0]), X, X, 2.5)
    assert r[0] == pytest.approx(t / (2.5 * (1 + t)), rel=1e-14)
    # left side enters through A^H and lambda^*: a complex eigenvalue and a
    # non-Hermitian A give different left/right residuals
    A = sp.csr_matrix(np.array([[1j, 1.0], [0.0, 2.0]]))
    Xr = np.array([[1.0], [0.0]], complex)          # exact right eigenvector of 1j
    Xl = np.array([[1.0], [t]], complex)
    r = F.residuals(A, None, np.array([1j]), Xr, Xl, 1.0)
    # A^H xl - conj(1j) xl = [-1j - (-1j), 1 + (2 + 1j) t]... computed by hand:
    Ah = A.toarray().conj().T
    v = Ah @ Xl[:, 0] - (-1j) * Xl[:, 0]
    assert v[0] == 0 and abs(v[1] - (1 + (2 + 1j) * t)) < 1e-15
    assert r[0] == pytest.approx(abs(1 + (2 + 1j) * t) / (1 + t), rel=1e-14)


@pytest.mark.parametrize("n,seed,cplx,withb", [(30, 1, True, True), (40, 2, True, False),
                                                (50, 3, False, True), (60, 4, False, False)])
def test_tiny_pencils_vs_qz(n, seed, cplx, withb):
    wk = wl.pencil_workload(n, seed, ne=8, m0=10, complex_=cplx, with_b=withb, n_inside=4)
    out = F.feast_nh(wk.A, wk.B, wk.contour, wk.m0, wk.Y0, wk.Yh0, eps=1e-10)
    assert out["converged"]
    ev = sla.eigvals(wk.A.toarray(), None if wk.B is None else wk.B.toarray())   # brute-force QZ
    ref = ev[inside(ev, wk.contour)]
    assert out["m"] == ref.size
    assert _match(out["lam"], ref) < 1e-9
    _invariants(wk, out)
    # right and left eigen-equations hold individually
    A = wk.A.toarray()
    B = np.eye(n) if wk.B is None else wk.B.toarray()
    for i in range(out["m"]):
        x, xh, l = out["X"][:, i], out["Xh"][:, i], out["lam"][i]
        assert np.linalg.norm(A @ x - l * B @ x) < 1e-8 * np.linalg.norm(x)
        assert np.linalg.norm(A.conj().T @ xh - np.conj(l) * B.conj().T @ xh) < 1e-8 * np.linalg.norm(xh)


def test_tridiag_symmetrised_closed_form_and_rate():
    # Symmetrised tridiagonal Toeplitz, circle |z-2| = 0.08: 36 eigenvalues
    # 2 + sqrt(2) cos(k pi/1001); the residual contracts at the rate
    # |rho_a(lambda_{m0+1}) / rho_a(lambda_m)| of Sec. 2.3.
    wk = wl.config1("b")
    out = F.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=False)
    assert out["converged"] and out["m"] == 36 == wk.exact.size
    assert np.max(np.abs(np.sort(out["lam"].real) - np.sort(wk.exact.real))) < 1e-12
    assert np.max(np.abs(out["lam"].imag)) < 1e-12
    _invariants(wk, out)
    z, w = contour_nodes(wk.contour)
    ev = wl.tridiag_toeplitz_eigs(1000, 1.0, 2.0, 0.5)
    r = np.sort(np.abs(rho_a(ev, z, w)))[::-1]
    predicted = r[wk.m0] / r[35]
    hist = [h["max_res"] for h in out["history"]]
    observed = (hist[29] / hist[19]) ** (1.0 / 10)     # asymptotic regime
    assert abs(observed / predicted - 1) < 0.01
    assert 25 <= out["iterations"] <= 40


def test_tridiag_nonnormal_small_closed_form():
    # The literal (unsymmetrised) matrix at n = 40: non-normal, eigenvalue condition ~1e5.
    wk = wl.config1("c")
    out = F.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=True, eps=1e-9)
    assert out["converged"] and out["m"] == wk.exact.size
    assert np.max(np.abs(np.sort(out["lam"].real) - np.sort(wk.exact.real))) < 1e-8


def test_convdiff_small_closed_form_and_gamma_identity():
    # 2D upwind convection-diffusion on 20x20 with an ellipse around 30 eigenvalues.
    wk = wl.config2(N=20, m0=48, ne=16)
    out = F.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=True, record=True)
    assert out["converged"] and out["m"] == 30
    assert _match(out["lam"], wk.exact) < 1e-10
    _invariants(wk, out)
    # eq. (bdiag1): from iteration 2 the eigenvalues of B_Q are rho_a^2 of the
    # previous Ritz values; compare the inside ones as multisets.
    h1, h2 = out["history"][-2], out["history"][-1]
    ins = inside(h1["lam"], wk.contour)
    r2 = h1["rho"][ins] ** 2
    dist = np.abs(h2["gamma"][None, :] - r2[:, None]).min(axis=1)
    assert np.max(dist) < 1e-6          # first order in the subspace error
    # Sec. 2.7: a Ritz value inside C that does not converge is flagged, so the
    # convergence test counts m = m_r - m_s = 30 genuine eigenvalues.
    assert h2["m_r"] - h2["m_s"] == 30 and out["history"][0]["m_s"] == 0


def test_spurious_identity_on_converged_pairs():
    # eq. (spurious0): [B_Q]_ii ~ rho_a^2(lambda_i) for genuine converged pairs,
    # so none of them is flagged; a perturbed diagonal is flagged.
    wk = wl.pencil_workload(40, 11, ne=8, m0=10)
    out = F.feast_nh(wk.A, wk.B, wk.contour, wk.m0, wk.Y0, wk.Yh0)
    z, w = contour_nodes(wk.contour)
    Y, Yh = out["Y"], out["Yh"]
    sol = F.node_solvers(wk.A, wk.B, z, True)
    Q, Qh = F.contour_integration(wk.A, wk.B, sol, z, w, Y, Yh)
    BQ = Qh.conj().T @ (wk.B @ Q)
    rho = rho_a(out["lam_all"], z, w)
    ins = inside(out["lam_all"], wk.contour)
    d = np.diag(BQ)
    assert np.max(np.abs(d[ins] - rho[ins] ** 2) / np.abs(rho[ins] ** 2)) < 1e-8
    assert not F.spurious_flags(BQ, rho)[ins].any()
    BQ2 = BQ.copy()
    k = np.where(ins)[0][0]
    BQ2[k, k] *= 1.2
    assert F.spurious_flags(BQ2, rho)[k]


def test_complex_symmetric_problem():
    # Sec. 2.4: complex symmetric A, B (3D Laplacian + absorbing layer, diagonal B):
    # X^ = conj(X); the shortcut Q^ = conj(Q) gives the same eigenvalues.
    A, B = wl.laplace3d_cap(6, 2)
    ev = sla.eigvals(A.toarray(), B.toarray())
    c = 1.2 - 0.05j
    d = np.sort(np.abs(ev - c))
    con = wl.Contour(0, c, 0.5 * (d[5] + d[6]), ne=16)
    ref = ev[inside(ev, con)]
    Y0 = wl.start_block(A.shape[0], 14, 0, complex_=True)
    out_g = F.feast_nh(A, B, con, 14, Y0, Y0.conj(), problem="general")
    out_c = F.feast_nh(A, B, con, 14, Y0, Y0.conj(), problem="complex_symmetric")
    for out in (out_g, out_c):
        assert out["converged"] and out["m"] == ref.size == 6
        assert _match(out["lam"], ref) < 1e-9
        X, Xh = out["X"], out["Xh"]
        cosang = np.abs(np.sum(Xh * X, axis=0)) / (np.linalg.norm(X, axis=0) * np.linalg.norm(Xh, axis=0))
        assert np.min(cosang) > 1 - 1e-9                      # x^_i parallel to conj(x_i)
        assert np.max(np.abs(Xh.conj().T @ (B @ X) - np.eye(6))) < 1e-10


def test_complex_symmetric_16cube_family_vs_arpack():
    # the config-3 family at 16^3 with 2 absorbing layers (Sec. 2.4, the CSH
    # stand-in): the oracle's eigenvalues inside the circle equal ARPACK's
    # shift-invert eigenvalues of the same pencil, none missing
    wk = wl.config3(L=16, layers=2, m0=32, ne=16, k_lo=16, k_hi=24, nev=40)
    out = F.feast_nh(wk.A, wk.B, wk.contour, wk.m0, wk.Y0, wk.Yh0, problem="complex_symmetric")
    assert out["converged"] and out["m"] == wk.exact.size >= 16
    assert _match(out["lam"], wk.exact) < 1e-10
    X, Xh = out["X"], out["Xh"]
    assert np.max(np.abs(Xh.conj().T @ (wk.B @ X) - np.eye(out["m"]))) < 1e-10
    cosang = np.abs(np.sum(Xh * X, axis=0)) / (np.linalg.norm(X, axis=0) * np.linalg.norm(Xh, axis=0))
    assert np.min(cosang) > 1 - 1e-9                          # x^_i parallel to conj(x_i)


@pytest.mark.parametrize("seed", [7, 8])
def test_random_sparse_family_vs_arpack(seed):
    # the many-problem family (random sparse, 9 entries a row, shifted
    # diagonal) at n < 1000 with its right-edge circle: the oracle finds every
    # eigenvalue ARPACK finds inside, to 1e-10
    bw = wl.config4(nprob=1, nmin=700, nmax=900, seed=seed, workers=1)
    A = bw.A[0]
    n = A.shape[0]
    out = F.feast_nh(A, None, bw.contours[0], bw.m0, bw.Y0[:n], bw.Yh0[:n])
    assert out["converged"] and out["m"] == bw.exact[0].size >= 16
    assert _match(out["lam"], bw.exact[0]) < 1e-10
    X, Xh = out["X"], out["Xh"]
    assert np.max(np.abs(Xh.conj().T @ X - np.eye(out["m"]))) < 1e-10


def test_resize_on_rank_deficient_start():
    # Duplicate start columns make B_Q singular: the subspace is resized
    # (eq. resize) and the run still converges.
    wk = wl.pencil_workload(40, 5, ne=8, m0=10)
    Y0 = wk.Y0.copy()
    Y0[:, 9] = Y0[:, 8]
    Yh0 = wk.Yh0.copy()
    Yh0[:, 9] = Yh0[:, 8]
    out = F.feast_nh(wk.A, wk.B, wk.contour, 10, Y0, Yh0, record=True)
    assert out["history"][0]["m_tilde"] == 9
    assert out["converged"] and out["m"] == wk.exact.size
    assert _match(out["lam"], wk.exact) < 1e-9
