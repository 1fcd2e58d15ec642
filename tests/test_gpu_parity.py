"""CUDA path (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from oracle import feast_nh as OF  # noqa: E402
from oracle.contour import contour_nodes, inside  # noqa: E402
from paper_1506_04463_gb300 import feast_nh as F  # noqa: E402
from paper_1506_04463_gb300 import workloads as wl  # noqa: E402
from gpu_helpers import dev, host, invariants, make_ctx, match_rel  # noqa: E402

PRECS = [F.PREC_FP64, F.PREC_FP32_IR]


def banded_workload(n=300, kl=5, ku=3, seed=0, m0=8, ne=8, with_b=True, pivoting=False):
    """Banded complex pencil in the class of the unpivoted banded solver
    (accretive shifted matrices, real positive diagonal B); pivoting=True
    gives a random banded pencil (complex diagonal B) that needs pivoting."""
    A = wl.banded_random(n, kl, ku, seed) if pivoting else wl.banded_accretive(n, kl, ku, seed)
    B = None
    if with_b:
        rng = np.random.default_rng(seed + 1)
        if pivoting:
            B = sp.diags(rng.uniform(1, 2, n) * np.exp(1j * rng.uniform(-0.2, 0.2, n))).tocsr()
        else:
            B = sp.diags(rng.uniform(1, 2, n) + 0j).tocsr()
    import scipy.linalg as sla
    ev = sla.eigvals(A.toarray(), None if B is None else B.toarray())
    c = np.median(ev.real) + 1j * np.median(ev.imag)
    d = np.sort(np.abs(ev - c))
    # radius across the widest relative gap with 3 .. m0 - 3 eigenvalues inside
    k = max(range(3, max(4, m0 - 2)), key=lambda k: (d[k] - d[k - 1]) / d[k])
    con = wl.Contour(0, complex(c), float(0.5 * (d[k - 1] + d[k])), ne=ne)
    return wl.Workload(f"banded{n}", A, B, con, m0, wl.start_block(n, m0, 0, True), wl.start_block(n, m0, 1, True),
                       "general", ev[np.abs(ev - c) <= con.r])


@pytest.mark.parametrize("prec", PRECS)
def test_multishift_residual_matches_definition(prec):
    wk = banded_workload(n=257, kl=4, ku=2, m0=7, ne=5)
    ctx = make_ctx(wk, precision=prec)
    z, w = contour_nodes(wk.contour)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((5, 257, 7)) + 1j * rng.standard_normal((5, 257, 7))
    BY = rng.standard_normal((257, 7)) + 1j * rng.standard_normal((257, 7))
    R, Q = ctx.multishift_residual(dev(X), dev(BY))
    Ro, Qo = OF.shifted_residuals(wk.A, wk.B, z, w, X, BY)
    assert np.max(np.abs(host(R) - Ro)) < 1e-12 * np.max(np.abs(Ro))
    assert np.max(np.abs(host(Q) - Qo)) < 1e-13 * np.max(np.abs(Qo))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["banded_B", "banded_noB", "pencil", "tridiag"])
def test_filter_matches_oracle(prec, case):
    if case == "banded_B":
        wk = banded_workload(n=300, kl=5, ku=3, with_b=True)
    elif case == "banded_noB":
        wk = banded_workload(n=161, kl=2, ku=7, with_b=False, m0=5, ne=6)
    elif case == "pencil":
        wk = wl.pencil_workload(40, 3, ne=8, m0=8)
    else:
        wk = wl.config1("b")
    ctx = make_ctx(wk, precision=prec)
    Q, Qh = ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    z, w = contour_nodes(wk.contour)
    Qo, Qho = OF.contour_integration(wk.A, wk.B, OF.node_solvers(wk.A, wk.B, z), z, w, wk.Y0, wk.Yh0)
    tol = 1e-10
    assert np.max(np.abs(host(Q) - Qo)) < tol * np.max(np.abs(Qo))
    assert np.max(np.abs(host(Qh) - Qho)) < tol * np.max(np.abs(Qho))


def test_rr_step_matches_oracle():
    wk = wl.pencil_workload(50, 4, ne=8, m0=10)
    z, w = contour_nodes(wk.contour)
    Qo, Qho = OF.contour_integration(wk.A, wk.B, OF.node_solvers(wk.A, wk.B, z), z, w, wk.Y0, wk.Yh0)
    ro = OF.rayleigh_ritz(wk.A, wk.B, Qo, Qho, z, w)
    ctx = make_ctx(wk)
    lam, Y, Yh, info = ctx.rr(dev(Qo), dev(Qho))
    assert info["m_tilde"] == ro["m_tilde"] == 10
    lam = host(lam)
    assert match_rel(lam, ro["lam"], 1e-3) < 1e-9
    # Ritz vectors agree up to scale: match by eigenvalue
    Y = host(Y)
    for i, l in enumerate(lam):
        k = np.argmin(np.abs(ro["lam"] - l))
        y, yo = Y[:, i], ro["Y"][:, k]
        assert abs(np.vdot(y, yo)) / (np.linalg.norm(y) * np.linalg.norm(yo)) > 1 - 1e-9
    # B-bi-orthonormal Ritz blocks (Y^^H B Y = I)
    BY = Y if wk.B is None else wk.B @ Y
    assert np.max(np.abs(host(Yh).conj().T @ BY - np.eye(10))) < 1e-10


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,seed,cplx,withb", [(30, 1, True, True), (40, 2, True, False), (50, 3, False, True),
                                                (61, 4, False, False)])
def test_solve_tiny_pencils(prec, n, seed, cplx, withb):
    wk = wl.pencil_workload(n, seed, ne=8, m0=10, complex_=cplx, with_b=withb, n_inside=4)
    oo = OF.feast_nh(wk.A, wk.B, wk.contour, wk.m0, wk.Y0, wk.Yh0)
    ctx = make_ctx(wk, precision=prec)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["status"] == F.OK and out["m"] == oo["m"] == wk.exact.size
    assert match_rel(host(out["lam"]), oo["lam"], 1e-3) < 1e-9
    invariants(wk, out)
    assert abs(out["info"]["iterations"] - oo["iterations"]) <= 2


@pytest.mark.parametrize("prec", PRECS)
def test_tridiagonal_closed_form(prec):
    wk = wl.config1("b")
    ctx = make_ctx(wk, precision=prec)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["status"] == F.OK and out["m"] == 36
    lam = np.sort(host(out["lam"]).real)
    assert np.max(np.abs(lam - np.sort(wk.exact.real))) < 1e-12
    assert np.max(np.abs(host(out["lam"]).imag)) < 1e-12
    invariants(wk, out)
    assert 28 <= out["info"]["iterations"] <= 34


@pytest.mark.parametrize("prec", PRECS)
def test_convdiff_closed_form(prec):
    wk = wl.config2(N=40, m0=48, ne=16)
    oo = OF.feast_nh(wk.A, None, wk.contour, wk.m0, wk.Y0, wk.Yh0, dense=False)
    ctx = make_ctx(wk, precision=prec)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["status"] == F.OK and out["m"] == 30 == oo["m"]
    assert match_rel(host(out["lam"]), wk.exact, 1e-3) < 1e-9
    assert match_rel(host(out["lam"]), oo["lam"], 1e-3) < 1e-9
    invariants(wk, out)


@pytest.mark.parametrize("mode", [F.PROBLEM_GENERAL, F.PROBLEM_COMPLEX_SYMMETRIC])
def test_complex_symmetric(mode):
    import scipy.linalg as sla
    A, B = wl.laplace3d_cap(6, 2)
    ev = sla.eigvals(A.toarray(), B.toarray())
    c = 1.2 - 0.05j
    d = np.sort(np.abs(ev - c))
    con = wl.Contour(0, c, 0.5 * (d[5] + d[6]), ne=16)
    Y0 = wl.start_block(A.shape[0], 14, 0, complex_=True)
    wk = wl.Workload("cap", A, B, con, 14, Y0, Y0.conj(), "complex_symmetric")
    ctx = F.FeastNH(A, B, con, 14, problem=mode)
    out = ctx.solve(dev(Y0), dev(Y0.conj()))
    assert out["status"] == F.OK and out["m"] == 6
    assert match_rel(host(out["lam"]), ev[inside(ev, con)], 1e-3) < 1e-9
    invariants(wk, out)
    X, Xh = host(out["X"]), host(out["Xh"])
    cosang = np.abs(np.sum(Xh * X, axis=0)) / (np.linalg.norm(X, axis=0) * np.linalg.norm(Xh, axis=0))
    assert np.min(cosang) > 1 - 1e-9


@pytest.mark.parametrize("prec", PRECS)
def test_config3_family_16cube(prec):
    # scaled member of the generalized complex-symmetric workload (16^3, two
    # absorbing layers, B diagonal; band 256): CUDA path vs oracle vs ARPACK
    wk = wl.config3(L=16, layers=2, m0=32, ne=16, k_lo=16, k_hi=24, nev=40)
    oo = OF.feast_nh(wk.A, wk.B, wk.contour, wk.m0, wk.Y0, wk.Yh0, problem="complex_symmetric")
    ctx = make_ctx(wk, precision=prec, problem=F.PROBLEM_COMPLEX_SYMMETRIC)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["status"] == F.OK and out["m"] == oo["m"] == wk.exact.size
    lam = host(out["lam"])
    assert match_rel(lam, oo["lam"], 1e-3) < 1e-9
    assert match_rel(lam, wk.exact, 1e-3) < 1e-9
    invariants(wk, out)
    X, Xh = host(out["X"]), host(out["Xh"])
    cosang = np.abs(np.sum(Xh * X, axis=0)) / (np.linalg.norm(X, axis=0) * np.linalg.norm(Xh, axis=0))
    assert np.min(cosang) > 1 - 1e-9
    assert abs(out["info"]["iterations"] - oo["iterations"]) <= 2
    ctx.close()


def test_edge_cases():
    # m0 = 1 with one eigenvalue inside; ne = 3; ragged n
    A = sp.diags(np.linspace(1.0, 2.0, 37) + 0j).tocsr()
    con = wl.Contour(0, 1.0 + 0j, 0.02, ne=3)
    Y0 = wl.start_block(37, 1, 0)
    ctx = F.FeastNH(A, None, con, 1)
    out = ctx.solve(dev(Y0), dev(Y0))
    assert out["m"] == 1 and abs(host(out["lam"])[0] - 1.0) < 1e-12


def test_node_on_eigenvalue_is_reported():
    # a quadrature node that coincides with an eigenvalue gives a zero pivot:
    # the library returns ESINGULAR (no fault)
    con = wl.Contour(0, 0j, 1.0, ne=4)
    z, _ = contour_nodes(con)
    d = np.array([z[0], 5.0, 6.0, 7.0, 8.0])
    A = sp.diags(d).tocsr()
    ctx = F.FeastNH(A, None, con, 2)
    Y0 = wl.start_block(5, 2, 0)
    with pytest.raises(F.FeastError) as e:
        ctx.solve(dev(Y0), dev(Y0))
    assert e.value.status == F.ESINGULAR


def test_determinism():
    wk = banded_workload(n=300, kl=5, ku=3)
    ctx = make_ctx(wk, precision=F.PREC_FP32_IR)
    a = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    b = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert torch.equal(a["lam"], b["lam"]) and torch.equal(a["X"], b["X"])


def _table_solve():
    import os
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table_solve_counts.txt")):
        if line.strip() and not line.startswith("#"):
            k, f, s = line.split()
            rows[k] = (float(f), float(s))
    return rows


def test_conjugate_pair_factorisation_count():
    # Table tab:solve: real non-symmetric with C = C^* needs ne/2
    # factorisations; complex general needs ne.  Results stay those of the oracle.
    rows = _table_solve()
    wk = wl.config2(N=30, m0=48, ne=16)
    ctx = make_ctx(wk, precision=F.PREC_FP32_IR)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["info"]["n_factorizations"] == rows["real_nonsymmetric_conj_contour"][0] * 16
    assert out["m"] == 30 and match_rel(host(out["lam"]), wk.exact, 1e-3) < 1e-9
    invariants(wk, out)
    # the same real pencil on a contour that is not symmetric about the real axis
    con = wl.Contour(0, complex(wk.contour.center) + 0.3 * wk.contour.r * 1j, wk.contour.r, ne=8)
    ctx2 = F.FeastNH(wk.A, None, con, wk.m0)
    out2 = ctx2.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out2["info"]["n_factorizations"] == 8
    wkc = banded_workload(n=300, kl=5, ku=3)
    ctx3 = make_ctx(wkc)
    out3 = ctx3.solve(dev(wkc.Y0), dev(wkc.Yh0))
    assert out3["info"]["n_factorizations"] == rows["complex_general"][0] * wkc.contour.ne


# ---------------- batched BiCGStab inner solver ----------------
def test_bicgstab_filter_matches_oracle():
    wk = wl.config1("b")
    ctx = make_ctx(wk, inner_kind=F.INNER_BICGSTAB, inner_max=4000, inner_tol=1e-12)
    Q, Qh = ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    z, w = contour_nodes(wk.contour)
    Qo, Qho = OF.contour_integration(wk.A, None, OF.node_solvers(wk.A, None, z, dense=False), z, w, wk.Y0, wk.Yh0)
    assert np.max(np.abs(host(Q) - Qo)) < 1e-9 * np.max(np.abs(Qo))
    assert np.max(np.abs(host(Qh) - Qho)) < 1e-9 * np.max(np.abs(Qho))


@pytest.mark.parametrize("case", ["pencil", "tridiag"])
def test_bicgstab_solve(case):
    if case == "pencil":
        wk = wl.pencil_workload(40, 3, ne=8, m0=8)
        oo = OF.feast_nh(wk.A, wk.B, wk.contour, wk.m0, wk.Y0, wk.Yh0)
        ref = oo["lam"]
    else:
        wk = wl.config1("b")
        ref = wk.exact
    ctx = make_ctx(wk, inner_kind=F.INNER_BICGSTAB, inner_max=4000, inner_tol=1e-12)
    out = ctx.solve(dev(wk.Y0), dev(wk.Yh0))
    assert out["status"] == F.OK and out["m"] == ref.size
    assert match_rel(host(out["lam"]), ref, 1e-3) < 1e-9
    invariants(wk, out)
    assert out["info"]["inner_steps"] > 1 and out["info"]["n_factorizations"] == 0


def test_bicgstab_reports_unconverged_interior_systems():
    # interior nodes of the convection-diffusion operator: Krylov stalls and the
    # filter reports FEAST_NH_EINNER (the banded direct solver handles these)
    wk = wl.config2(N=30, m0=48, ne=16)
    ctx = make_ctx(wk, inner_kind=F.INNER_BICGSTAB, inner_max=60, inner_tol=1e-12)
    with pytest.raises(F.FeastError) as e:
        ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    assert e.value.status == F.EINNER


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["banded_B", "banded_noB"])
def test_pivoting_needed_is_reported(prec, case):
    # random complex banded pencils need pivoting at interior shifts; the
    # unpivoted banded solver does not pivot, and the refinement residual
    # reports the inaccurate solves as FEAST_NH_EINNER instead of a silent result
    if case == "banded_B":
        wk = banded_workload(n=300, kl=5, ku=3, with_b=True, pivoting=True)
    else:
        wk = banded_workload(n=161, kl=2, ku=7, with_b=False, m0=5, ne=6, pivoting=True)
    ctx = make_ctx(wk, precision=prec)
    with pytest.raises(F.FeastError) as e:
        ctx.filter(dev(wk.Y0), dev(wk.Yh0))
    assert e.value.status == F.EINNER
    ctx.close()
