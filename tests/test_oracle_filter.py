"""Pins of the oracle's contour integration (eq. qr, eq. ql, Sec. 2.4)."""
import os

import numpy as np
import scipy.sparse as sp

from oracle import feast_nh as F
from oracle.contour import rho_a, trapezoid_nodes
from paper_1506_04463_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


def _blocks(n, m, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    Yh = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    return Y, Yh


def test_diagonal_pencil_is_rho_a_scaling():
    # (z B - A)^{-1} B = diag(1/(z - a_i/b_i)) for diagonal A, B: Q = diag(rho_a(l_i)) Y
    # and Q^ = diag(conj(rho_a(l_i))) Y^ exactly (eq. q00, eq. qhat0).
    n, m = 30, 5
    rng = np.random.default_rng(1)
    a = rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)
    b = rng.uniform(0.5, 2, n) * np.exp(1j * rng.uniform(-0.5, 0.5, n))
    A, B = sp.diags(a).tocsr(), sp.diags(b).tocsr()
    z, w = trapezoid_nodes(0.1 + 0.2j, 0.6, 1.0, 0.0, 8)
    Y, Yh = _blocks(n, m, 2)
    for dense in (True, False):
        Q, Qh = F.contour_integration(A, B, F.node_solvers(A, B, z, dense), z, w, Y, Yh)
        r = rho_a(a / b, z, w)
        assert np.max(np.abs(Q - r[:, None] * Y)) < 1e-12
        assert np.max(np.abs(Qh - np.conj(r)[:, None] * Yh)) < 1e-12


def test_filter_matches_spectral_form():
    # Q = X rho_a(L) X^{-1} Y with B^{-1}A = X L X^{-1}; Q^ = rho_a(A B^{-1})^H Y^ with
    # rho_a(A B^{-1}) = B X rho_a(L) X^{-1} B^{-1} (eq. q00, eq. qhat0).
    wk = wl.pencil_workload(24, 7, ne=8, m0=4)
    A, B = wk.A.toarray(), wk.B.toarray()
    z, w = trapezoid_nodes(wk.contour.center, wk.contour.r, 1.0, 0.0, 8)
    lam, X = np.linalg.eig(np.linalg.solve(B, A))
    R = X @ np.diag(rho_a(lam, z, w)) @ np.linalg.inv(X)
    Y, Yh = _blocks(24, 4, 3)
    Q, Qh = F.contour_integration(wk.A, wk.B, F.node_solvers(wk.A, wk.B, z, True), z, w, Y, Yh)
    assert np.max(np.abs(Q - R @ Y)) < 1e-10 * np.max(np.abs(Q))
    Rl = B @ R @ np.linalg.inv(B)
    assert np.max(np.abs(Qh - Rl.conj().T @ Yh)) < 1e-10 * np.max(np.abs(Qh))


def test_complex_symmetric_shortcut():
    # Sec. 2.4: A = A^T, B = B^T  =>  Q^ = conj(Q) when Y^ = conj(Y).
    A, B = wl.laplace3d_cap(5, 2)
    z, w = trapezoid_nodes(2.0 - 0.1j, 0.4, 1.0, 0.0, 8)
    Y, _ = _blocks(A.shape[0], 3, 4)
    sol = F.node_solvers(A, B, z, True)
    Qg, Qhg = F.contour_integration(A, B, sol, z, w, Y, Y.conj(), "general")
    Qc, Qhc = F.contour_integration(A, B, sol, z, w, Y, Y.conj(), "complex_symmetric")
    assert np.max(np.abs(Qg - Qc)) == 0
    assert np.max(np.abs(Qhg - Qhc)) < 1e-12 * np.max(np.abs(Qhg))


def test_solve_counts_match_paper_table():
    # Table tab:solve: factorizations / solves per full contour integration.
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table_solve_counts.txt")):
        if line.strip() and not line.startswith("#"):
            k, f, s = line.split()
            rows[k] = (float(f), float(s))

    class Counting(F.NodeSolver):
        solves = 0
        facts = 0

        def __init__(self, *a, **k):
            Counting.facts += 1
            super().__init__(*a, **k)

        def solve(self, rhs, herm=False):
            Counting.solves += 1
            return super().solve(rhs, herm)

    ne = 8
    for fam, problem in (("complex_general", "general"), ("complex_symmetric", "complex_symmetric")):
        Counting.solves = Counting.facts = 0
        A, B = wl.laplace3d_cap(4, 1)
        z, w = trapezoid_nodes(1.0, 0.5, 1.0, 0.0, ne)
        sol = [Counting(A, B, zj, True) for zj in z]
        Y, _ = _blocks(A.shape[0], 2, 5)
        F.contour_integration(A, B, sol, z, w, Y, Y.conj(), problem)
        assert (Counting.facts, Counting.solves) == (rows[fam][0] * ne, rows[fam][1] * ne)
