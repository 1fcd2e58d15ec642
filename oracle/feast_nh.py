"""Non-Hermitian FEAST, plain FP64 on the CPU (oracle; test infrastructure only).

Follows the complete algorithm of Fig. alg:three step by step:
  0  start blocks Y, Y^ (given)
  1  contour integration, eq. (qr) and eq. (ql)
  2  B_Q = Q^^H B Q and the spurious test of Sec. 2.7
  3  B_Q = V Gamma V^^H, resize (eq. resize), B-bi-orthonormal U, U^ (eq. uu)
  4  Rayleigh-Ritz on U, U^ (QZ), rho_a of the Ritz values, Ritz vectors
  5  convergence test on eq. (res), converged pairs placed first.

Readings where the paper is silent (each listed in the design notes):
  * the left Ritz block is W^ = (W^{-1} B_U^{-1})^H, which is the left
    eigenvector block of the pencil (A_U, B_U) scaled so that W^^H B_U W = I;
  * V^^H = V^{-1} for B_Q = V Gamma V^^H (so that V^^H V = I);
  * Gamma^{-1/2} uses the principal square root, Gamma^{-H/2} its conjugate;
  * sort by |gamma| is stable (ties keep their index order);
  * Ritz vectors are scaled to ||y_i||_2 = 1 with y^_i^H B y_i unchanged;
  * the spurious test compares [B_Q]_ii of this iteration with rho_a^2 of
    the previous Ritz value i; m_s counts flagged values that were inside;
  * the loop stops when the m = m_r - m_s lowest inside residuals are below
    eps; it then returns every inside pair with residual below eps (a genuine
    pair flagged from a not-yet-converged previous iterate is kept);
  * complex symmetric problems use Q^ = conj(Q), V^ = conj(V), W^ = conj(W)
    with v^T v = 1 and w^T B_U w = 1 (Sec. 2.4), so that Y^ = conj(Y).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .contour import alpha as contour_alpha
from .contour import contour_nodes, inside, rho_a


def _mat(M):
    return M


class NodeSolver:
    """LU of (z_j B - A) for one quadrature node, reused for the conjugate-
    transpose solve (Sec. 2.4: one factorisation serves eq. (qr) and eq. (ql))
    and across iterations (the saved-factorisation option of Sec. 4.1)."""

    def __init__(self, A, B, zj, dense: bool):
        n = A.shape[0]
        Bm = sp.identity(n, dtype=np.complex128, format="csr") if B is None else B
        M = (zj * Bm - A)
        self.dense = dense
        if dense:
            Md = M.toarray() if sp.issparse(M) else np.asarray(M)
            self.lu = sla.lu_factor(Md.astype(np.complex128))
        else:
            self.lu = spla.splu(sp.csc_matrix(M, dtype=np.complex128))

    def solve(self, rhs, herm: bool = False):
        rhs = np.asarray(rhs, np.complex128)
        if self.dense:
            return sla.lu_solve(self.lu, rhs, trans=2 if herm else 0)
        return self.lu.solve(rhs, trans="H" if herm else "N")


def node_solvers(A, B, z, dense=None):
    n = A.shape[0]
    if dense is None:
        dense = n <= 2000
    return [NodeSolver(A, B, zj, dense) for zj in z]


def _B(B, X):
    return X if B is None else B @ X


def _BH(B, X):
    return X if B is None else B.conj().T @ X


def _solve_each(solvers, rhs, herm):
    """(z_j B - A)^{-1} rhs (or ^{-H}) for every node j, in node order.  A
    solver list may instead provide solve_all(rhs, herm) returning the same
    list (e.g. one worker process per node); the sums below are unchanged."""
    if hasattr(solvers, "solve_all"):
        return solvers.solve_all(rhs, herm)
    return [s.solve(rhs, herm=herm) for s in solvers]


def contour_integration(A, B, solvers, z, w, Y, Yh, problem="general"):
    """Step 1: Q = sum_j w_j (z_j B - A)^{-1} B Y            (eq. qr)
               Q^ = sum_j w_j^* (z_j B - A)^{-H} B^H Y^      (eq. ql)
    Complex symmetric: Q^ = conj(Q) (Sec. 2.4), valid for Y^ = conj(Y)."""
    BY = _B(B, Y)
    Q = np.zeros(Y.shape, np.complex128)
    for j, Xj in enumerate(_solve_each(solvers, BY, False)):
        Q += w[j] * Xj
    if problem == "complex_symmetric":
        return Q, Q.conj()
    BhYh = _BH(B, Yh)
    Qh = np.zeros(Yh.shape, np.complex128)
    for j, Xj in enumerate(_solve_each(solvers, BhYh, True)):
        Qh += np.conj(w[j]) * Xj
    return Q, Qh


def spurious_flags(BQ, rho_prev, mu=0.1):
    """Step 2.b (Sec. 2.7): flag i if |(rho_a^2(lambda_i) - [B_Q]_ii)/rho_a^2(lambda_i)| >= mu."""
    r2 = np.asarray(rho_prev, np.complex128) ** 2
    d = np.diag(BQ)[: r2.size]
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.abs((r2 - d) / r2)
    return ~(q < mu)


def rayleigh_ritz(A, B, Q, Qh, z, w, eta=1e-16, problem="general"):
    """Steps 2.a, 3 and 4 of Fig. alg:three."""
    cs = problem == "complex_symmetric"
    BQ = Qh.conj().T @ _B(B, Q)                                   # 2.a
    gam, V = np.linalg.eig(BQ)                                    # 3.a
    order = np.argsort(-np.abs(gam), kind="stable")               # 3.c
    gam, V = gam[order], V[:, order]
    if cs:
        V = V / np.sqrt(np.sum(V * V, axis=0))
        VhH = V.T                                                 # V^^H = conj(V)^H
    else:
        VhH = np.linalg.inv(V)                                    # V^^H V = I
    gmax = np.max(np.abs(gam))
    mt = int(np.sum(np.abs(gam) >= eta * gmax))                   # 3.b, eq. (resize)
    s = 1.0 / np.sqrt(gam[:mt])                                   # Gamma^{-1/2}
    U = (Q @ V[:, :mt]) * s[None, :]                              # 3.d, eq. (uu)
    Uh = (Qh @ VhH[:mt, :].conj().T) * np.conj(s)[None, :]
    BU = Uh.conj().T @ _B(B, U)                                   # 4.a
    AU = Uh.conj().T @ (A @ U)
    lam, W = sla.eig(AU, BU)                                      # 4.b (QZ)
    if cs:
        W = W / np.sqrt(np.sum(W * (BU @ W), axis=0))
        Wh = W.conj()
    else:
        W = W / np.linalg.norm(W, axis=0)
        Wh = (np.linalg.inv(W) @ np.linalg.inv(BU)).conj().T      # W^^H B_U W = I
    rho = rho_a(lam, z, w)                                        # 4.c
    Y = U @ W                                                     # 4.d
    Yh = Uh @ Wh
    if not cs:
        # Only W^^H B_U W = I is fixed by the method; the free column scale is
        # set to ||y_i||_2 = 1 (y^_i rescaled so that y^_i^H B y_i is kept), so
        # that the column scales of Y and Y^ cannot drift apart over iterations.
        nrm = np.linalg.norm(Y, axis=0)
        Y = Y / nrm[None, :]
        Yh = Yh * nrm[None, :]
    return dict(lam=lam, Y=Y, Yh=Yh, rho=rho, BQ=BQ, gamma=gam, m_tilde=mt, BU=BU, AU=AU)


def residuals(A, B, lam, X, Xh, alpha):
    """eq. (res): max(||A x - lambda B x||_1 / ||alpha B x||_1,
                      ||A^H x^ - lambda^* B^H x^||_1 / ||alpha B^H x^||_1)."""
    lam = np.asarray(lam, np.complex128)
    BX = _B(B, X)
    r1 = np.abs(A @ X - BX * lam[None, :]).sum(0) / (alpha * np.abs(BX).sum(0))
    BhXh = _BH(B, Xh)
    AhXh = A.conj().T @ Xh
    r2 = np.abs(AhXh - BhXh * np.conj(lam)[None, :]).sum(0) / (alpha * np.abs(BhXh).sum(0))
    return np.maximum(r1, r2)


def normalize_pairs(B, X, Xh):
    """Output scaling: ||x_i||_2 = 1 with its largest-modulus entry real
    positive; x^_i scaled so that x^_i^H B x_i = 1."""
    X = X.copy()
    Xh = Xh.copy()
    for i in range(X.shape[1]):
        k = np.argmax(np.abs(X[:, i]))
        ph = X[k, i] / abs(X[k, i])
        X[:, i] /= ph * np.linalg.norm(X[:, i])
        t = np.vdot(Xh[:, i], _B(B, X[:, i]))
        Xh[:, i] /= np.conj(t)
    return X, Xh


def feast_nh(A, B, con, m0, Y0, Yh0, eps=1e-10, eta=1e-16, mu=0.1, max_iter=100,
             problem="general", dense=None, solvers=None, record=False):
    """The complete non-Hermitian FEAST algorithm (Fig. alg:three).

    Returns a dict with lam (m), X, Xh (n x m), res (m), m, iterations,
    converged, and per-iteration history.
    """
    z, w = contour_nodes(con)
    alpha = contour_alpha(con)
    if solvers is None:
        solvers = node_solvers(A, B, z, dense)
    Y = np.asarray(Y0, np.complex128)[:, :m0]
    Yh = np.asarray(Yh0, np.complex128)[:, :m0]
    if problem == "complex_symmetric":
        Yh = Y.conj()
    rho_prev = None
    ins_prev = None
    hist = []
    out = None
    for it in range(1, max_iter + 1):
        Q, Qh = contour_integration(A, B, solvers, z, w, Y, Yh, problem)      # 1
        rr = rayleigh_ritz(A, B, Q, Qh, z, w, eta, problem)                    # 2.a, 3, 4
        m_s = 0
        if it >= 2:                                                            # 2.b
            fl = spurious_flags(rr["BQ"], rho_prev, mu)
            m_s = int(np.sum(fl & ins_prev))
        lam, Y, Yh = rr["lam"], rr["Y"], rr["Yh"]
        ins = inside(lam, con)                                                 # 5.a
        m_r = int(ins.sum())
        res = np.full(lam.shape, np.inf)
        if m_r:
            res[ins] = residuals(A, B, lam[ins], Y[:, ins], Yh[:, ins], alpha)  # 5.b
        m = m_r - m_s
        idx = np.where(ins)[0]
        idx = idx[np.argsort(res[idx], kind="stable")]
        top = idx[: max(m, 0)]
        conv = m >= 1 and bool(np.all(res[top] < eps))                        # 5.c
        h = dict(it=it, m_tilde=rr["m_tilde"], m_r=m_r, m_s=m_s,
                 max_res=float(np.max(res[top])) if m >= 1 else float("inf"))
        if conv:
            # 5.d: every inside pair whose residual is below eps is returned
            # (spurious values do not converge, Sec. 2.7), at least m of them
            top = idx[res[idx] < eps]
        if record:
            h.update(gamma=rr["gamma"], rho=rr["rho"], lam=lam, res=res)
        hist.append(h)
        rho_prev, ins_prev = rr["rho"], ins
        if conv or it == max_iter:
            X, Xh = normalize_pairs(B, Y[:, top], Yh[:, top])                   # 5.d
            out = dict(lam=lam[top], X=X, Xh=Xh, res=res[top], m=len(top), iterations=it,
                       converged=conv, history=hist, Y=Y, Yh=Yh, lam_all=lam, res_all=res)
            break
    return out


def shifted_residuals(A, B, z, w, X, BY):
    """Plain definition of the residuals of the shifted systems of eq. (qr):
    R_j = B Y - (z_j B - A) X_j for every node j, and Q = sum_j w_j X_j.
    X: (ne, n, m) array; BY: (n, m)."""
    R = np.empty_like(X)
    Q = np.zeros(X.shape[1:], np.complex128)
    for j in range(len(z)):
        BX = _B(B, X[j])
        R[j] = BY - (z[j] * BX - A @ X[j])
        Q += w[j] * X[j]
    return R, Q
