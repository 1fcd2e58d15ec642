"""Seeded synthetic inputs for the non-Hermitian FEAST filter and Rayleigh-Ritz.

This module builds matrices, contours and start blocks only.  It holds none of
the method's arithmetic (no quadrature, no filter, no Rayleigh-Ritz); both the
CUDA path and the CPU oracle take their inputs from here.

Every workload stands in for a data set of the paper that is not available
(the NEP collection, CSH4, the dense unit-disk matrix of Sec. 4): the shapes,
sparsity and spectra below are synthetic and seeded.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Contour:
    """Circle (kind 0) or ellipse (kind 1) of Sec. 2.1, or custom nodes (kind 2).

    Ellipse: centre c, horizontal semi-axis r, vertical semi-axis ratio*r,
    rotated by `angle` radians.  A circle is the ellipse with ratio 1, angle 0.
    """
    kind: int
    center: complex
    r: float
    ratio: float = 1.0
    angle: float = 0.0
    ne: int = 8
    z: np.ndarray | None = None      # custom nodes (kind 2)
    w: np.ndarray | None = None      # custom weights (kind 2)


@dataclass
class Workload:
    name: str
    A: sp.csr_matrix
    B: sp.csr_matrix | None           # None = identity
    contour: Contour
    m0: int
    Y0: np.ndarray                    # n x m0, right start block
    Yh0: np.ndarray                   # n x m0, left start block
    problem: str = "general"          # general | complex_symmetric | real
    exact: np.ndarray | None = None   # closed-form eigenvalues inside the contour
    meta: dict = field(default_factory=dict)


def start_block(n: int, m0: int, seed: int, complex_: bool = False) -> np.ndarray:
    """Random start subspace (step 0 of the complete algorithm): N(0,1) entries,
    or (N(0,1) + i N(0,1))/sqrt(2) for complex problems; column-major n x m0."""
    rng = np.random.default_rng(seed)
    if complex_:
        y = (rng.standard_normal((n, m0)) + 1j * rng.standard_normal((n, m0))) / math.sqrt(2.0)
    else:
        y = rng.standard_normal((n, m0)).astype(np.complex128)
    return np.asfortranarray(y)


def tridiag_toeplitz(n: int, sub: float, diag: float, sup: float) -> sp.csr_matrix:
    e = np.ones(n)
    return sp.diags([sub * e[1:], diag * e, sup * e[1:]], [-1, 0, 1], format="csr")


def tridiag_toeplitz_eigs(n: int, sub: float, diag: float, sup: float) -> np.ndarray:
    """Closed form: diag + 2 sqrt(sub*sup) cos(k pi/(n+1)), k = 1..n."""
    k = np.arange(1, n + 1)
    return diag + 2.0 * np.sqrt(complex(sub * sup)) * np.cos(k * np.pi / (n + 1))


def symmetrized_tridiag(n: int, sub: float, diag: float, sup: float):
    """Diagonal similarity D^{-1} A D of a tridiagonal Toeplitz matrix with
    d_1 = 1, d_{i+1} = d_i sqrt(sub/sup): off-diagonals become sqrt(sub*sup).
    Right eigenvectors map back by x = D x~, left ones by x^ = D^{-1} x^~."""
    s = math.sqrt(sub * sup)
    A = tridiag_toeplitz(n, s, diag, s)
    logd = np.arange(n) * 0.5 * math.log(sub / sup)
    return A, logd


def config1(variant: str = "b", m0: int = 40, ne: int = 8) -> Workload:
    """Tridiagonal Toeplitz (sub 1.0, diag 2.0, super 0.5), n = 1000, circle
    |z - 2| = 0.08, B = I.  Variant 'a' is the literal matrix, 'b' its
    symmetrised similarity (the solved matrix), 'c' the literal matrix at n = 40
    with a circle around the 6 eigenvalues nearest 2."""
    if variant == "c":
        n = 40
        A = tridiag_toeplitz(n, 1.0, 2.0, 0.5)
        ev = tridiag_toeplitz_eigs(n, 1.0, 2.0, 0.5).real
        con = Contour(0, 2.0 + 0j, 0.3, ne=ne)
        m0 = min(m0, 12)
    else:
        n = 1000
        if variant == "a":
            A = tridiag_toeplitz(n, 1.0, 2.0, 0.5)
        else:
            A, _ = symmetrized_tridiag(n, 1.0, 2.0, 0.5)
        ev = tridiag_toeplitz_eigs(n, 1.0, 2.0, 0.5).real
        con = Contour(0, 2.0 + 0j, 0.08, ne=ne)
    inside = np.sort(ev[np.abs(ev - con.center) <= con.r])
    return Workload(f"tridiag_toeplitz_n{n}_{variant}", A.tocsr(), None, con, m0,
                    start_block(n, m0, 0), start_block(n, m0, 1), "real",
                    inside.astype(np.complex128))


def convdiff2d(N: int, beta: float = 10.0) -> sp.csr_matrix:
    """-Lap u + beta du/dx on the unit square, Dirichlet, first-order upwind,
    scaled by h^2: diag 4+g, x-sub -(1+g), x-super -1, y-neighbours -1,
    g = beta*h, x the fastest index."""
    h = 1.0 / (N + 1)
    g = beta * h
    e = np.ones(N)
    Tx = sp.diags([-(1 + g) * e[1:], (2 + g) * e, -e[1:]], [-1, 0, 1])
    Ty = sp.diags([-e[1:], 2 * e, -e[1:]], [-1, 0, 1])
    I = sp.identity(N)
    return (sp.kron(I, Tx) + sp.kron(Ty, I)).tocsr()


def convdiff2d_eigs(N: int, beta: float = 10.0) -> np.ndarray:
    """Closed form (2+g) - 2 sqrt(1+g) cos(k pi/(N+1)) + 2 - 2 cos(l pi/(N+1)), sorted."""
    h = 1.0 / (N + 1)
    g = beta * h
    k = np.arange(1, N + 1)
    lx = (2 + g) - 2 * np.sqrt(1 + g) * np.cos(k * np.pi / (N + 1))
    ly = 2 - 2 * np.cos(k * np.pi / (N + 1))
    return np.sort((lx[:, None] + ly[None, :]).ravel())


def config2(N: int = 300, beta: float = 10.0, m: int = 30, m0: int = 64, ne: int = 16,
            start_lo: int | None = None) -> Workload:
    """2D convection-diffusion (Peclet 10 upwind), ellipse (ratio 0.5, angle 0)
    around m consecutive closed-form eigenvalues; the first index is chosen in
    [start_lo, start_lo+100) to maximise the smaller outer gap, and the
    horizontal semi-axis is half the span plus half that gap."""
    A = convdiff2d(N, beta)
    lam = convdiff2d_eigs(N, beta)
    n = N * N
    if start_lo is None:
        start_lo = 300 if n > 4000 else max(1, n // 4)
    best = None
    for s in range(start_lo, min(start_lo + 100, n - m - 1)):
        gap = min(lam[s] - lam[s - 1], lam[s + m] - lam[s + m - 1])
        if best is None or gap > best[0]:
            best = (gap, s)
    gap, s = best
    lo, hi = lam[s], lam[s + m - 1]
    c = 0.5 * (lo + hi)
    a = 0.5 * (hi - lo) + 0.5 * gap
    con = Contour(1, complex(c), a, ratio=0.5, angle=0.0, ne=ne)
    return Workload(f"convdiff2d_N{N}", A, None, con, m0, start_block(n, m0, 0),
                    start_block(n, m0, 1), "real", lam[s:s + m].astype(np.complex128),
                    {"N": N, "beta": beta, "first_index": s, "gap": gap})


def laplace3d_cap(L: int, layers: int, seed_cap: int = 0, seed_b: int = 1):
    """7-point Laplacian (diag 6, off -1, Dirichlet) on L^3 plus i*U(-0.5,0) on
    sites within `layers` of a face; B = diag(U(1,2)).  Complex symmetric."""
    e = np.ones(L)
    T = sp.diags([-e[1:], 2 * e, -e[1:]], [-1, 0, 1])
    I = sp.identity(L)
    A = (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).tocsr()
    idx = np.arange(L)
    edge = (idx < layers) | (idx >= L - layers)
    ex, ey, ez = np.meshgrid(edge, edge, edge, indexing="ij")
    absorb = (ex | ey | ez).ravel()
    rng = np.random.default_rng(seed_cap)
    cap = np.where(absorb, rng.uniform(-0.5, 0.0, L ** 3), 0.0)
    A = (A.astype(np.complex128) + sp.diags(1j * cap)).tocsr()
    rngb = np.random.default_rng(seed_b)
    B = sp.diags(rngb.uniform(1.0, 2.0, L ** 3)).tocsr().astype(np.complex128)
    return A, B


def nearest_circle(A, B, target: complex, k_lo: int, k_hi: int, nev: int):
    """Circle centred at `target` holding k_lo..k_hi eigenvalues of the pencil
    (A, B) (input construction only: ARPACK shift-invert, the `nev` eigenvalues
    nearest the target).  Radius halfway across the widest relative gap among
    the sorted distances; every eigenvalue inside is among the computed ones.
    Returns (contour, eigenvalues inside)."""
    import scipy.sparse.linalg as spla
    ev = spla.eigs(A.tocsc(), k=nev, M=None if B is None else B.tocsc(), sigma=target, which="LM",
                   return_eigenvectors=False, tol=1e-13)
    d = np.sort(np.abs(ev - target))
    best = None
    for k in range(k_lo, min(k_hi, nev - 1) + 1):
        r = 0.5 * (d[k - 1] + d[k])
        gap = (d[k] - d[k - 1]) / r
        if best is None or gap > best[0]:
            best = (gap, r)
    r = best[1]
    con = Contour(0, complex(target), r)
    return con, np.sort_complex(ev[np.abs(ev - target) <= r])


def config3(L: int = 64, layers: int = 8, m0: int = 128, ne: int = 16, target: complex = 0.35 - 0.1j,
            k_lo: int = 40, k_hi: int = 60, nev: int = 80) -> Workload:
    """Generalized complex-symmetric problem: 7-point Laplacian on L^3 plus an
    absorbing potential i*U(-0.5, 0) on the outer `layers` layers, B = diag
    U(1, 2); a circle around k_lo..k_hi eigenvalues nearest `target`; complex
    start block (N(0,1) + iN(0,1))/sqrt(2), Yh0 = conj(Y0) (Sec. 2.4).  The
    full size is L = 64, layers = 8, m0 = 128, 40-60 eigenvalues; L = 16,
    layers = 2 is the scaled family member a banded solver reaches."""
    A, B = laplace3d_cap(L, layers)
    con, ev = nearest_circle(A, B, target, k_lo, k_hi, nev)
    con = Contour(0, con.center, con.r, ne=ne)
    Y0 = start_block(A.shape[0], m0, 0, complex_=True)
    return Workload(f"laplace3d_cap_{L}", A, B, con, m0, Y0, Y0.conj(), "complex_symmetric", exact=ev,
                    meta={"L": L, "layers": layers})


def random_sparse(n: int, seed: int, nnz_row: int = 9, shift_max: float = 4.0) -> sp.csr_matrix:
    """Each row: the diagonal plus nnz_row-1 distinct random off-diagonal
    columns, values N(0, 1/9); then diagonal += U(0, shift_max)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        c = rng.choice(n - 1, size=nnz_row - 1, replace=False)
        c = c + (c >= i)
        rows.append(np.full(nnz_row, i))
        cols.append(np.concatenate(([i], c)))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = rng.normal(0.0, 1.0 / 3.0, rows.size)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A = A + sp.diags(rng.uniform(0.0, shift_max, n))
    return A.tocsr()


def random_pencil(n: int, seed: int, complex_: bool = True, with_b: bool = True):
    """Small dense general pencil (A, B) with B = I + 0.1 N(0,1) (well conditioned)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    if complex_:
        A = A + 1j * rng.standard_normal((n, n))
    A = A / math.sqrt(n)
    B = None
    if with_b:
        B = np.eye(n) + 0.1 * rng.standard_normal((n, n)) / math.sqrt(n)
        if complex_:
            B = B + 0.1j * rng.standard_normal((n, n)) / math.sqrt(n)
    return sp.csr_matrix(A.astype(np.complex128)), (None if B is None else sp.csr_matrix(B.astype(np.complex128)))


def banded_random(n: int, kl: int, ku: int, seed: int, complex_: bool = True) -> sp.csr_matrix:
    """Random banded matrix (kl sub-, ku super-diagonals), N(0,1) entries."""
    rng = np.random.default_rng(seed)
    diags, offs = [], []
    for d in range(-kl, ku + 1):
        m = n - abs(d)
        v = rng.standard_normal(m)
        if complex_:
            v = v + 1j * rng.standard_normal(m)
        diags.append(v)
        offs.append(d)
    return sp.diags(diags, offs, format="csr").astype(np.complex128)


def banded_accretive(n: int, kl: int, ku: int, seed: int, complex_: bool = True) -> sp.csr_matrix:
    """Banded matrix that Gaussian elimination without pivoting factors
    stably at any non-real shift: A = S^{-1} H S with H Hermitian banded
    (half-bandwidth min(kl, ku), N(0,1) entries scaled by 1/sqrt(band)) and
    S = diag(exp(U(-1/2, 1/2))); the wider side of an unequal band gets
    extra diagonals of size 1e-3.  Then z I - A = S^{-1}(z I - H) S and every
    pivot of z I - H has |Im pivot| >= |Im z| > 0."""
    rng = np.random.default_rng(seed)
    k = min(kl, ku)
    H = np.zeros((n, n), np.complex128)
    H[np.arange(n), np.arange(n)] = rng.standard_normal(n)
    for d in range(1, k + 1):
        v = rng.standard_normal(n - d) / math.sqrt(k)
        if complex_:
            v = v + 1j * rng.standard_normal(n - d) / math.sqrt(k)
        H[np.arange(n - d), np.arange(d, n)] = v
        H[np.arange(d, n), np.arange(n - d)] = np.conj(v)
    for d in range(k + 1, max(kl, ku) + 1):
        v = 1e-3 * rng.standard_normal(n - d)
        if ku > kl:
            H[np.arange(n - d), np.arange(d, n)] = v
        else:
            H[np.arange(d, n), np.arange(n - d)] = v
    s = np.exp(rng.uniform(-0.5, 0.5, n))
    A = (H / s[:, None]) * s[None, :]
    if not complex_:
        A = A.real
    return sp.csr_matrix(A.astype(np.complex128))


def pencil_workload(n: int, seed: int, ne: int = 8, m0: int = 8, complex_: bool = True,
                    with_b: bool = True, n_inside: int = 3) -> Workload:
    """Tiny dense pencil with a circle around the (at least) n_inside eigenvalues
    nearest the spectrum's centroid; the radius sits halfway across the first
    gap of at least 10% that follows them.
    Eigenvalues of the pencil are needed to place the contour (input
    construction only)."""
    import scipy.linalg as sla
    A, B = random_pencil(n, seed, complex_, with_b)
    ev = sla.eigvals(A.toarray(), None if B is None else B.toarray())
    c = np.mean(ev)
    d = np.sort(np.abs(ev - c))
    # the circle passes through a gap of at least 10% of the radius, so that no
    # eigenvalue (e.g. one of a conjugate pair) lies on or near the contour
    k = n_inside
    while k < n - 1 and d[k] - d[k - 1] < 0.1 * d[k]:
        k += 1
    r = 0.5 * (d[k - 1] + d[k])
    con = Contour(0, complex(c), float(r), ne=ne)
    return Workload(f"pencil_n{n}_s{seed}", A, B, con, m0,
                    start_block(n, m0, 2 * seed, complex_), start_block(n, m0, 2 * seed + 1, complex_),
                    "general", np.sort_complex(ev[np.abs(ev - c) <= r]))


def edge_circle(A: sp.csr_matrix, k_lo: int = 16, k_hi: int = 40, nev: int = 48, seed: int = 0):
    """Circle around eigenvalues at the right edge of the spectrum of a real
    sparse A (input construction only: ARPACK's `nev` rightmost eigenvalues).
    Centre on the real axis just right of the rightmost eigenvalue; radius
    halfway across the widest relative gap among the sorted distances with
    k_lo..k_hi eigenvalues inside, and small enough that every eigenvalue it
    can hold is among the computed ones.  Returns (contour, eigenvalues
    inside)."""
    import scipy.sparse.linalg as spla
    n = A.shape[0]
    v0 = np.random.default_rng(seed).standard_normal(n)
    ev = spla.eigs(A.astype(np.float64), k=nev, which="LR", return_eigenvectors=False, tol=1e-12, v0=v0,
                   ncv=min(n, max(2 * nev + 1, 120)))
    ev = ev[np.argsort(-ev.real)]
    c = float(ev[0].real) + 0.02
    d = np.sort(np.abs(ev - c))
    lo_bound = c - float(ev[-1].real)          # a radius beyond this could hold uncomputed eigenvalues
    best = None
    for k in range(k_lo, min(k_hi, nev - 1) + 1):
        r = 0.5 * (d[k - 1] + d[k])
        gap = (d[k] - d[k - 1]) / r
        if r < 0.95 * lo_bound and (best is None or gap > best[0]):
            best = (gap, r)
    if best is None:
        raise ValueError("no radius with 16..40 computed eigenvalues inside")
    r = best[1]
    con = Contour(0, complex(c), r)
    return con, np.sort_complex(ev[np.abs(ev - c) <= r])


@dataclass
class BatchWorkload:
    name: str
    A: list                      # per-problem CSR matrices (B = I)
    contours: list               # per-problem Contour
    m0: int
    Y0: np.ndarray               # (sum n_p) x m0, problems stacked by rows
    Yh0: np.ndarray
    exact: list                  # per-problem eigenvalues inside (ARPACK, for checks)
    offsets: np.ndarray          # first row of each problem


def _config4_problem(args):
    p, n, m0 = args
    Ap = random_sparse(n, 100 + p)
    con, inside = edge_circle(Ap, seed=p)
    return Ap, con, inside, start_block(n, m0, 2 * p), start_block(n, m0, 2 * p + 1)


def config4(nprob: int = 64, nmin: int = 5000, nmax: int = 200000, m0: int = 48, ne: int = 8,
            seed: int = 0, workers: int | None = None) -> BatchWorkload:
    """Many independent random sparse nonsymmetric problems: sizes log-uniform
    in [nmin, nmax] (seed), rows as random_sparse (seed 100 + p), B = I, each
    with its own circle at the right edge of its spectrum holding 16..40
    eigenvalues, m0 columns, ne trapezoid nodes; start blocks N(0,1) with
    seeds 2p and 2p + 1.  `workers` > 1 builds the problems in that many
    spawned processes (same result)."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(math.log(nmin), math.log(nmax), nprob))).astype(int)
    args = [(p, int(n), m0) for p, n in enumerate(sizes)]
    if workers and workers > 1 and nprob > 1:
        import multiprocessing as mp
        import os
        from concurrent.futures import ProcessPoolExecutor
        # one BLAS thread per worker process: the workers already fill the cores
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            with ProcessPoolExecutor(max_workers=min(workers, nprob), mp_context=mp.get_context("spawn")) as ex_:
                parts = list(ex_.map(_config4_problem, args))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    else:
        parts = [_config4_problem(a) for a in args]
    A, cons, ex, Y, Yh = [], [], [], [], []
    for Ap, con, inside, y, yh in parts:
        con.ne = ne
        A.append(Ap)
        cons.append(con)
        ex.append(inside)
        Y.append(y)
        Yh.append(yh)
    offs = np.concatenate(([0], np.cumsum(sizes)[:-1]))
    return BatchWorkload(f"random_sparse_batch{nprob}", A, cons, m0, np.ascontiguousarray(np.vstack(Y)),
                         np.ascontiguousarray(np.vstack(Yh)), ex, offs)
