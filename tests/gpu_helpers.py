"""Shared helpers of the GPU parity tests (CUDA path vs oracle)."""
import numpy as np
import torch
from scipy.optimize import linear_sum_assignment

from paper_1506_04463_gb300 import feast_nh as F


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.complex128))).cuda()


def host(t):
    return t.detach().cpu().numpy()


def match_rel(a, b, floor):
    """Max |a_i - b_pi(i)| / max(|b|, floor) after optimal one-to-one matching."""
    a, b = np.asarray(a), np.asarray(b)
    assert a.size == b.size, (a.size, b.size)
    if a.size == 0:
        return 0.0
    Cm = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(Cm)
    return float(np.max(Cm[r, c] / np.maximum(np.abs(b[c]), floor)))


def make_ctx(wk, **opts):
    return F.FeastNH(wk.A, wk.B, wk.contour, wk.m0, **opts)


def invariants(wk, out, tol_bi=1e-10, tol_res=1e-10):
    from oracle.contour import inside
    from oracle.feast_nh import residuals
    from oracle.contour import alpha
    X, Xh, lam = host(out["X"]), host(out["Xh"]), host(out["lam"])
    BX = X if wk.B is None else wk.B @ X
    assert np.max(np.abs(Xh.conj().T @ BX - np.eye(X.shape[1]))) < tol_bi
    assert np.all(inside(lam, wk.contour))
    r = residuals(wk.A, wk.B, lam, X, Xh, alpha(wk.contour))
    assert np.all(r < tol_res), r.max()
    # the residuals the library reports are eq. (res) as well
    assert np.allclose(host(out["res"]), r, rtol=1e-3, atol=1e-14)
    return r
