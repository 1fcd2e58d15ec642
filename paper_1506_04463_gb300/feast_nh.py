"""Python binding of the C ABI in include/feast_nh.h (argument marshalling only).

Every numerical step runs in libfeast_nh.so.  If the library is missing the
binding raises; there is no fallback path.  Device memory and streams come
from PyTorch.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfeast_nh.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EINNER, ESINGULAR, ETIMEOUT = range(8)
DEVERR_ZERO_PIVOT, DEVERR_QR_NOCONV, DEVERR_TIMEOUT = 1, 2, 16
R64, C64 = 0, 1
INNER_BANDED, INNER_BICGSTAB, INNER_FGMRES = 0, 1, 2
PRECOND_NONE, PRECOND_JACOBI, PRECOND_LEARNED = 0, 1, 2
PREC_FP64, PREC_FP32_IR = 0, 1
PROJ_FP64, PROJ_TENSOR = 0, 1
PROBLEM_GENERAL, PROBLEM_COMPLEX_SYMMETRIC = 0, 1


class Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("val", C.c_void_p), ("dtype", C.c_int32)]


class ContourS(C.Structure):
    _fields_ = [("kind", C.c_int32), ("c_re", C.c_double), ("c_im", C.c_double), ("r", C.c_double),
                ("ratio", C.c_double), ("angle", C.c_double), ("ne", C.c_int32),
                ("z", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double))]


class Opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("eta", C.c_double), ("mu", C.c_double), ("inner_tol", C.c_double),
                ("max_iter", C.c_int32), ("inner_max", C.c_int32), ("inner_kind", C.c_int32),
                ("precision", C.c_int32), ("problem", C.c_int32), ("timing", C.c_int32),
                ("krylov_max", C.c_int32), ("krylov_restart", C.c_int32), ("precond", C.c_int32),
                ("projection", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("m_tilde", C.c_int32), ("m_r", C.c_int32), ("m_s", C.c_int32),
                ("m", C.c_int32), ("inner_steps", C.c_int32), ("converged", C.c_int32), ("kl", C.c_int32),
                ("ku", C.c_int32), ("max_res", C.c_double), ("inner_res", C.c_double),
                ("t_factor_ms", C.c_double), ("t_filter_ms", C.c_double), ("t_rr_ms", C.c_double),
                ("t_total_ms", C.c_double), ("t_solve_kernel_ms", C.c_double), ("t_resid_kernel_ms", C.c_double),
                ("n_solve_launches", C.c_int32), ("n_resid_launches", C.c_int32), ("n_factorizations", C.c_int32),
                ("inner_fail", C.c_int32), ("pivot_min", C.c_double), ("pivot_max", C.c_double),
                ("krylov_iterations", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged_problems", C.c_int32), ("inner_fail", C.c_int32),
                ("krylov_iterations", C.c_int32), ("refine_steps", C.c_int32), ("threads", C.c_int32),
                ("tile_rows", C.c_int32), ("grid", C.c_int32), ("max_res", C.c_double), ("inner_res", C.c_double),
                ("t_filter_ms", C.c_double), ("t_rr_ms", C.c_double), ("t_total_ms", C.c_double),
                ("t_autotune_ms", C.c_double), ("graph", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["feast_nh_default_opts", "feast_nh_init", "feast_nh_filter", "feast_nh_rr", "feast_nh_solve",
           "feast_nh_destroy", "feast_nh_strerror", "feast_nh_last_error", "feast_nh_nodes",
           "feast_nh_multishift_residual", "feast_nh_kernel_launches", "feast_nh_multishift_residual_noalloc",
           "feast_nh_small_eig", "feast_nh_inject_device_error", "feast_nh_batch_init", "feast_nh_batch_solve",
           "feast_nh_batch_destroy", "feast_nh_batch_last_error", "feast_nh_multishift_spmm", "feast_nh_net_create",
           "feast_nh_net_set_params", "feast_nh_net_get_params", "feast_nh_net_forward", "feast_nh_net_train_step",
           "feast_nh_net_destroy", "feast_nh_net_last_error", "feast_nh_set_network", "feast_nh_learned_pairs",
           "feast_nh_operator_loss", "feast_nh_net_backward", "feast_nh_gram",
           "feast_nh_block_product", "feast_nh_release_memory"]

_lib = None


def lib():
    """Load libfeast_nh.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1506_04463_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32 = C.c_void_p, C.c_int32
    L.feast_nh_default_opts.argtypes = [C.POINTER(Opts)]
    L.feast_nh_default_opts.restype = None
    L.feast_nh_init.argtypes = [C.POINTER(vp), C.POINTER(Csr), C.POINTER(Csr), C.POINTER(ContourS), i32,
                                C.POINTER(Opts), vp]
    L.feast_nh_filter.argtypes = [vp, vp, vp, vp, vp, i32]
    L.feast_nh_rr.argtypes = [vp, vp, vp, i32, vp, vp, vp, C.POINTER(i32), C.POINTER(Info)]
    L.feast_nh_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(i32), C.POINTER(Info)]
    L.feast_nh_destroy.argtypes = [vp]
    L.feast_nh_destroy.restype = None
    L.feast_nh_strerror.argtypes = [i32]
    L.feast_nh_strerror.restype = C.c_char_p
    L.feast_nh_last_error.argtypes = [vp]
    L.feast_nh_last_error.restype = C.c_char_p
    L.feast_nh_nodes.argtypes = [C.POINTER(ContourS), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.feast_nh_multishift_residual.argtypes = [vp, vp, vp, vp, vp, i32, i32]
    L.feast_nh_small_eig.argtypes = [vp, vp, i32, vp, vp]
    L.feast_nh_gram.argtypes = [vp, vp, vp, i32, i32, vp, i32]
    L.feast_nh_release_memory.argtypes = []
    L.feast_nh_release_memory.restype = i32
    L.feast_nh_block_product.argtypes = [vp, vp, vp, i32, i32, vp, i32]
    L.feast_nh_multishift_spmm.argtypes = [vp, vp, vp, i32, i32]
    L.feast_nh_inject_device_error.argtypes = [vp, C.c_uint32]
    L.feast_nh_multishift_residual_noalloc.argtypes = [C.POINTER(Csr), C.POINTER(Csr), C.POINTER(ContourS), vp, vp,
                                                       vp, vp, vp, i32, vp]
    L.feast_nh_multishift_residual_noalloc.restype = i32
    L.feast_nh_batch_init.argtypes = [C.POINTER(vp), i32, C.POINTER(Csr), C.POINTER(ContourS), i32, C.POINTER(Opts),
                                      vp]
    L.feast_nh_batch_init.restype = i32
    L.feast_nh_batch_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(BatchInfo)]
    L.feast_nh_batch_solve.restype = i32
    L.feast_nh_batch_destroy.argtypes = [vp]
    L.feast_nh_batch_destroy.restype = None
    L.feast_nh_batch_last_error.argtypes = [vp]
    L.feast_nh_batch_last_error.restype = C.c_char_p
    L.feast_nh_net_create.argtypes = [C.POINTER(vp), i32, i32, i32, vp]
    L.feast_nh_net_set_params.argtypes = [vp, C.POINTER(C.c_float)]
    L.feast_nh_net_get_params.argtypes = [vp, C.POINTER(C.c_float)]
    L.feast_nh_net_forward.argtypes = [vp, vp, vp, i32]
    L.feast_nh_net_train_step.argtypes = [vp, vp, vp, i32, i32, C.c_float, C.POINTER(C.c_double), vp]
    L.feast_nh_net_destroy.argtypes = [vp]
    L.feast_nh_net_destroy.restype = None
    L.feast_nh_net_last_error.argtypes = [vp]
    L.feast_nh_net_last_error.restype = C.c_char_p
    for f in ("feast_nh_net_create", "feast_nh_net_set_params", "feast_nh_net_get_params", "feast_nh_net_forward",
              "feast_nh_net_train_step"):
        getattr(L, f).restype = i32
    L.feast_nh_set_network.argtypes = [vp, vp, i32, C.c_float, C.POINTER(C.c_float), i32]
    L.feast_nh_set_network.restype = i32
    L.feast_nh_learned_pairs.argtypes = [vp, vp, i32, i32, C.c_float, C.POINTER(C.c_float), i32, vp, vp]
    L.feast_nh_learned_pairs.restype = i32
    L.feast_nh_operator_loss.argtypes = [vp, vp, vp, i32, i32, i32, vp, C.POINTER(C.c_double)]
    L.feast_nh_operator_loss.restype = i32
    L.feast_nh_net_backward.argtypes = [vp, vp, i32, C.c_float, vp]
    L.feast_nh_net_backward.restype = i32
    L.feast_nh_kernel_launches.argtypes = []
    L.feast_nh_kernel_launches.restype = C.c_uint64
    for f in ("feast_nh_init", "feast_nh_filter", "feast_nh_rr", "feast_nh_solve", "feast_nh_nodes",
              "feast_nh_multishift_residual", "feast_nh_small_eig", "feast_nh_inject_device_error",
              "feast_nh_multishift_spmm", "feast_nh_gram", "feast_nh_block_product"):
        getattr(L, f).restype = i32
    _lib = L
    return L


class FeastError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib().feast_nh_strerror(status).decode()}: {msg}")
        self.status = status


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().feast_nh_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def contour_struct(con) -> tuple[ContourS, list]:
    """Marshal a workloads.Contour (or any object with the same fields)."""
    keep = []
    s = ContourS()
    s.kind = int(con.kind)
    s.c_re, s.c_im = float(complex(con.center).real), float(complex(con.center).imag)
    s.r = float(con.r)
    s.ratio = float(getattr(con, "ratio", 1.0))
    s.angle = float(getattr(con, "angle", 0.0))
    s.ne = int(con.ne if con.kind != 2 else len(con.z))
    if con.kind == 2:
        z = np.ascontiguousarray(np.asarray(con.z, np.complex128)).view(np.float64)
        w = np.ascontiguousarray(np.asarray(con.w, np.complex128)).view(np.float64)
        keep += [z, w]
        s.z = z.ctypes.data_as(C.POINTER(C.c_double))
        s.w = w.ctypes.data_as(C.POINTER(C.c_double))
    return s, keep


def kernel_launches() -> int:
    """Kernels libfeast_nh.so has launched in this process."""
    return int(lib().feast_nh_kernel_launches())


def release_memory():
    """Give the library's reserved (unused) device workspace back to the
    driver; contexts and batches reuse it otherwise."""
    st = lib().feast_nh_release_memory()
    if st != OK:
        raise FeastError(st, "feast_nh_release_memory")


def multishift_residual_noalloc(A_dev, B_dev, contour, X, BY, want_q=True, stream=None):
    """feast_nh_multishift_residual_noalloc: R, Q and relative column norms
    with no context and no device allocation inside the library (the output
    tensors are allocated here by the caller).

    X: (ne, n, m) and BY: (n, m), contiguous complex128 on the device that
    holds the CSR arrays; the call runs with that device current, on `stream`
    (default: its current stream)."""
    if X.dtype != torch.complex128 or BY.dtype != torch.complex128:
        raise TypeError("X and BY must be complex128")
    if X.dim() != 3 or BY.dim() != 2:
        raise ValueError("X must be (ne, n, m) and BY (n, m)")
    if not (X.is_contiguous() and BY.is_contiguous()):
        raise ValueError("X and BY must be contiguous (the kernels read them after this call returns)")
    ne, n, m = X.shape
    cs, keep = contour_struct(contour)
    if ne != cs.ne or BY.shape != (n, m) or n != A_dev[4] or (B_dev is not None and B_dev[4] != n):
        raise ValueError(f"shape mismatch: X {tuple(X.shape)}, BY {tuple(BY.shape)}, n={A_dev[4]}, ne={cs.ne}")
    devs = {X.device, BY.device, A_dev[0].device, A_dev[2].device}
    if B_dev is not None:
        devs |= {B_dev[0].device, B_dev[2].device}
    if len(devs) != 1 or X.device.type != "cuda":
        raise ValueError("all operands must be on the same CUDA device")
    with torch.cuda.device(X.device):
        R = torch.empty_like(X)
        Q = torch.empty((n, m), dtype=torch.complex128, device=X.device) if want_q else None
        rel = torch.empty(ne * m, dtype=torch.float64, device=X.device)
        a = _csr_struct(A_dev)
        b = _csr_struct(B_dev) if B_dev is not None else None
        st = stream if stream is not None else torch.cuda.current_stream(X.device)
        rc = lib().feast_nh_multishift_residual_noalloc(C.byref(a), C.byref(b) if b is not None else None,
                                                        C.byref(cs), _ptr(X), _ptr(BY), _ptr(R), _ptr(Q), _ptr(rel),
                                                        m, C.c_void_p(st.cuda_stream))
        if rc != OK:
            raise FeastError(rc, "feast_nh_multishift_residual_noalloc")
        if st != torch.cuda.current_stream(X.device):
            # the caching allocator must not hand these blocks out again before
            # the kernels on `st` have used them
            for t in (X, BY, R, Q, rel):
                if t is not None:
                    t.record_stream(st)
    return R, Q, rel.view(ne, m)


def nodes(con):
    """Quadrature nodes/weights exactly as the library computes them."""
    s, keep = contour_struct(con)
    z = np.zeros(2 * s.ne)
    w = np.zeros(2 * s.ne)
    st = lib().feast_nh_nodes(C.byref(s), z.ctypes.data_as(C.POINTER(C.c_double)),
                              w.ctypes.data_as(C.POINTER(C.c_double)))
    if st != OK:
        raise FeastError(st, "feast_nh_nodes")
    return z.view(np.complex128), w.view(np.complex128)


def csr_to_device(M, device="cuda"):
    """Upload a scipy CSR matrix as int32 rowptr/colind and float64/complex128 values."""
    M = M.tocsr()
    rp = torch.from_numpy(M.indptr.astype(np.int32)).to(device)
    ci = torch.from_numpy(M.indices.astype(np.int32)).to(device)
    if np.iscomplexobj(M.data) and np.any(M.data.imag != 0):
        val = torch.from_numpy(np.ascontiguousarray(M.data.astype(np.complex128))).to(device)
        dt = C64
    else:
        val = torch.from_numpy(np.ascontiguousarray(M.data.real.astype(np.float64))).to(device)
        dt = R64
    return (rp, ci, val, dt, M.shape[0], M.nnz)


def _csr_struct(t) -> Csr:
    rp, ci, val, dt, n, nnz = t
    return Csr(n, nnz, rp.data_ptr(), ci.data_ptr(), val.data_ptr(), dt)


def _ptr(t):
    return None if t is None else t.data_ptr()


class FeastNH:
    """One context of the C ABI: pencil (A, B), contour, subspace size m0."""

    def __init__(self, A, B, contour, m0, device="cuda", stream=None, **opts):
        L = lib()
        self.device = torch.device(device)
        self.A_dev = A if isinstance(A, tuple) else csr_to_device(A, self.device)
        self.B_dev = None if B is None else (B if isinstance(B, tuple) else csr_to_device(B, self.device))
        self.n = self.A_dev[4]
        self.m0 = int(m0)
        self.opts = default_opts(**opts)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cs, self._keep = contour_struct(contour)
        self.ne = cs.ne
        a = _csr_struct(self.A_dev)
        b = _csr_struct(self.B_dev) if self.B_dev is not None else None
        h = C.c_void_p()
        st = L.feast_nh_init(C.byref(h), C.byref(a), C.byref(b) if b is not None else None, C.byref(cs),
                             self.m0, C.byref(self.opts), C.c_void_p(self.stream.cuda_stream))
        if st != OK:
            raise FeastError(st, "feast_nh_init (see argument checks)")
        self.h = h

    def _check(self, st, what, ok=(OK, ENOCONV)):
        if st not in ok:
            raise FeastError(st, f"{what}: {lib().feast_nh_last_error(self.h).decode()}")
        return st

    def _blk(self, m):
        return torch.empty((self.n, m), dtype=torch.complex128, device=self.device)

    def filter(self, Y, Yh=None):
        m = Y.shape[1]
        Q, Qh = self._blk(m), self._blk(m)
        st = lib().feast_nh_filter(self.h, _ptr(Y.contiguous()), _ptr(None if Yh is None else Yh.contiguous()),
                                   _ptr(Q), _ptr(Qh), m)
        self._check(st, "feast_nh_filter")
        return Q, Qh

    def rr(self, Q, Qh):
        m = Q.shape[1]
        lam = torch.empty(m, dtype=torch.complex128, device=self.device)
        Y, Yh = self._blk(m), self._blk(m)
        mn = C.c_int32()
        info = Info()
        st = lib().feast_nh_rr(self.h, _ptr(Q.contiguous()), _ptr(Qh.contiguous()), m, _ptr(lam), _ptr(Y),
                               _ptr(Yh), C.byref(mn), C.byref(info))
        self._check(st, "feast_nh_rr")
        k = mn.value
        # Y, Yh hold n x k row-major blocks with leading dimension k
        Yk = Y.view(-1)[: self.n * k].view(self.n, k)
        Yhk = Yh.view(-1)[: self.n * k].view(self.n, k)
        return lam[:k], Yk, Yhk, info.as_dict()

    def solve(self, Y0, Yh0=None):
        lam = torch.zeros(self.m0, dtype=torch.complex128, device=self.device)
        res = torch.zeros(self.m0, dtype=torch.float64, device=self.device)
        X, Xh = self._blk(self.m0), self._blk(self.m0)
        mf = C.c_int32()
        info = Info()
        st = lib().feast_nh_solve(self.h, _ptr(Y0.contiguous()), _ptr(None if Yh0 is None else Yh0.contiguous()),
                                  _ptr(lam), _ptr(X), _ptr(Xh), _ptr(res), C.byref(mf), C.byref(info))
        # ENOCONV / EINNER: the outputs hold the best iterate, the status says why
        self._check(st, "feast_nh_solve", ok=(OK, ENOCONV, EINNER))
        m = mf.value
        return dict(status=st, lam=lam[:m], X=X[:, :m], Xh=Xh[:, :m], res=res[:m], m=m, info=info.as_dict())

    def multishift_residual(self, X, BY, want_q=True, r_single=False):
        ne, n, m = X.shape
        R = torch.empty(X.shape, dtype=torch.complex64 if r_single else torch.complex128, device=X.device)
        Q = self._blk(m) if want_q else None
        Xc, BYc = X.contiguous(), BY.contiguous()
        st = lib().feast_nh_multishift_residual(self.h, _ptr(Xc), _ptr(BYc), _ptr(R), _ptr(Q), m,
                                                1 if r_single else 0)
        self._check(st, "feast_nh_multishift_residual")
        self.stream.synchronize()
        return R, Q

    def multishift_spmm(self, P, side=0, out=None):
        """Single-precision multi-shift operator: V_j = (z_j B - A) P_j (side 0)
        or (conj z_j B^H - A^H) P_j (side 1); P: (ne, n, m) complex64."""
        if P.dtype != torch.complex64 or not P.is_contiguous():
            raise TypeError("P must be a contiguous complex64 tensor")
        V = torch.empty_like(P) if out is None else out
        st = lib().feast_nh_multishift_spmm(self.h, _ptr(P), _ptr(V), P.shape[2], int(side))
        self._check(st, "feast_nh_multishift_spmm")
        return V

    def small_eig(self, M):
        """Eigenvalues and right eigenvectors of an m x m complex matrix by the
        library's small dense eigensolver (device tensors)."""
        m = M.shape[0]
        Mc = M.to(torch.complex128).contiguous()
        lam = torch.empty(m, dtype=torch.complex128, device=M.device)
        V = torch.empty((m, m), dtype=torch.complex128, device=M.device)
        st = lib().feast_nh_small_eig(self.h, _ptr(Mc), m, _ptr(lam), _ptr(V))
        self._check(st, "feast_nh_small_eig")
        return lam, V

    def gram(self, X, Y, method=None):
        """G = X^H Y (X: n x mx, Y: n x my device tensors) by the library's
        projection kernels; method PROJ_TENSOR (default) or PROJ_FP64."""
        Xc = X.to(torch.complex128).contiguous()
        Yc = Y.to(torch.complex128).contiguous()
        if Xc.shape[0] != self.n or Yc.shape[0] != self.n:
            raise ValueError("gram: X and Y need n rows")
        mx, my = Xc.shape[1], Yc.shape[1]
        G = torch.empty((mx, my), dtype=torch.complex128, device=Xc.device)
        st = lib().feast_nh_gram(self.h, _ptr(Xc), _ptr(Yc), mx, my, _ptr(G),
                                 PROJ_TENSOR if method is None else method)
        self._check(st, "feast_nh_gram")
        return G

    def block_product(self, X, S, method=None):
        """Z = X S (X: n x mx, S: mx x mz device tensors) by the library's
        block-update kernels; method PROJ_TENSOR (default) or PROJ_FP64."""
        Xc = X.to(torch.complex128).contiguous()
        Sc = S.to(device=Xc.device, dtype=torch.complex128).contiguous()
        if Xc.shape[0] != self.n or Sc.shape[0] != Xc.shape[1]:
            raise ValueError("block_product: X must be n x mx and S mx x mz")
        mx, mz = Sc.shape
        Z = torch.empty((self.n, mz), dtype=torch.complex128, device=Xc.device)
        st = lib().feast_nh_block_product(self.h, _ptr(Xc), _ptr(Sc), mx, mz, _ptr(Z),
                                          PROJ_TENSOR if method is None else method)
        self._check(st, "feast_nh_block_product")
        return Z

    def learned_pairs(self, R, N, kappa=1.0, features=()):
        """(inputs, targets) for the network from exact solves of R (n x m):
        (ne*m, N, N, 32) and (ne*m, N, N, 2) float32 device tensors."""
        Rc = R.to(torch.complex128).contiguous()
        m = Rc.shape[1]
        S = self.ne * m
        Xin = torch.empty((S, N, N, NET_CH), dtype=torch.float32, device=self.device)
        T = torch.empty((S, N, N, 2), dtype=torch.float32, device=self.device)
        f = np.ascontiguousarray(np.asarray(features, np.float32))
        st = lib().feast_nh_learned_pairs(self.h, _ptr(Rc), m, int(N), float(kappa),
                                          f.ctypes.data_as(C.POINTER(C.c_float)) if f.size else None, int(f.size),
                                          _ptr(Xin), _ptr(T))
        self._check(st, "feast_nh_learned_pairs")
        return Xin, T

    def operator_loss(self, out, T, N, side=0):
        """Operator-norm loss of network outputs against exact corrections and
        its gradient with respect to the outputs."""
        out, T = out.contiguous(), T.contiguous()
        m = out.shape[0] // self.ne
        g = torch.empty_like(out)
        loss = C.c_double()
        st = lib().feast_nh_operator_loss(self.h, _ptr(out), _ptr(T), m, int(N), int(side), _ptr(g), C.byref(loss))
        self._check(st, "feast_nh_operator_loss")
        return loss.value, g

    def set_network(self, net, N, kappa=1.0, features=()):
        """Attach a trained Net as the FGMRES right preconditioner."""
        f = np.ascontiguousarray(np.asarray(features, np.float32))
        self._net = net  # the context does not own the network; keep it alive
        st = lib().feast_nh_set_network(self.h, net.h, int(N), float(kappa),
                                        f.ctypes.data_as(C.POINTER(C.c_float)) if f.size else None, int(f.size))
        self._check(st, "feast_nh_set_network")

    def inject_device_error(self, bits):
        """Host-side fault injection: the next filter ORs `bits` into the
        device error word (no device fault is made)."""
        st = lib().feast_nh_inject_device_error(self.h, int(bits))
        self._check(st, "feast_nh_inject_device_error")

    def close(self):
        if getattr(self, "h", None):
            lib().feast_nh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FeastBatch:
    """Many independent standard problems (B = I) solved together: one
    persistent launch for the contour integration of all of them, the
    Rayleigh-Ritz steps concurrently (feast_nh_batch_* of the C ABI).

    A: list of scipy CSR matrices (or device tuples from csr_to_device);
    contours: one per problem, all with the same ne."""

    def __init__(self, A, contours, m0, device="cuda", stream=None, **opts):
        L = lib()
        self.device = torch.device(device)
        self.A_dev = [a if isinstance(a, tuple) else csr_to_device(a, self.device) for a in A]
        self.sizes = [a[4] for a in self.A_dev]
        self.offsets = np.concatenate(([0], np.cumsum(self.sizes)[:-1])).astype(np.int64)
        self.ntot = int(sum(self.sizes))
        self.nprob = len(self.A_dev)
        self.m0 = int(m0)
        opts.setdefault("inner_kind", INNER_BICGSTAB)
        self.opts = default_opts(**opts)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        csrs = (Csr * self.nprob)(*[_csr_struct(a) for a in self.A_dev])
        self._keep = []
        cons = (ContourS * self.nprob)()
        for p, c in enumerate(contours):
            cs, keep = contour_struct(c)
            cons[p] = cs
            self._keep += keep
        h = C.c_void_p()
        st = L.feast_nh_batch_init(C.byref(h), self.nprob, csrs, cons, self.m0, C.byref(self.opts),
                                   C.c_void_p(self.stream.cuda_stream))
        if st != OK:
            raise FeastError(st, "feast_nh_batch_init")
        self.h = h

    def solve(self, Y0, Yh0):
        """Y0, Yh0: (sum n_p, m0) complex128 device tensors.  Returns per-problem
        lists of eigenvalues, residuals, X, Xh views and the info dict."""
        n, m0, P = self.ntot, self.m0, self.nprob
        lam = torch.zeros(P * m0, dtype=torch.complex128, device=self.device)
        res = torch.zeros(P * m0, dtype=torch.float64, device=self.device)
        X = torch.zeros((n, m0), dtype=torch.complex128, device=self.device)
        Xh = torch.zeros((n, m0), dtype=torch.complex128, device=self.device)
        mf = (C.c_int32 * P)()
        its = (C.c_int32 * P)()
        info = BatchInfo()
        Y0c, Yh0c = Y0.contiguous(), Yh0.contiguous()
        st = lib().feast_nh_batch_solve(self.h, _ptr(Y0c), _ptr(Yh0c), _ptr(lam), _ptr(X), _ptr(Xh), _ptr(res), mf,
                                        its, C.byref(info))
        if st not in (OK, ENOCONV, EINNER):
            raise FeastError(st, "feast_nh_batch_solve: " + lib().feast_nh_batch_last_error(self.h).decode())
        out = []
        for p in range(P):
            o, npb, m = int(self.offsets[p]), self.sizes[p], mf[p]
            # problem p's block: rows [o, o + n_p) of the (sum n_p, m0) arrays
            out.append(dict(lam=lam[p * m0: p * m0 + m], res=res[p * m0: p * m0 + m], X=X[o:o + npb, :m],
                            Xh=Xh[o:o + npb, :m], m=m, iterations=its[p]))
        return dict(status=st, problems=out, info=info.as_dict())

    def close(self):
        if getattr(self, "h", None):
            lib().feast_nh_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NET_CH = 32
NET_LAYER_PARAMS = 9 * NET_CH * NET_CH + NET_CH


class Net:
    """The learned preconditioner's network (feast_nh_net_* of the C ABI):
    `layers` 3x3 convolutions, 32 channels, on an N x N grid."""

    def __init__(self, layers, N, max_images, device="cuda", stream=None):
        self.layers, self.N, self.max_images = int(layers), int(N), int(max_images)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = lib().feast_nh_net_create(C.byref(h), self.layers, self.N, self.max_images,
                                       C.c_void_p(self.stream.cuda_stream))
        if st != OK:
            raise FeastError(st, "feast_nh_net_create")
        self.h = h

    def _check(self, st, what):
        if st != OK:
            raise FeastError(st, f"{what}: {lib().feast_nh_net_last_error(self.h).decode()}")

    def set_params(self, params):
        p = np.ascontiguousarray(np.asarray(params, np.float32).ravel())
        assert p.size == self.layers * NET_LAYER_PARAMS
        self._check(lib().feast_nh_net_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))), "set_params")

    def get_params(self):
        p = np.zeros(self.layers * NET_LAYER_PARAMS, np.float32)
        self._check(lib().feast_nh_net_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))), "get_params")
        return p

    def forward(self, x):
        """x: (nimg, N, N, 32) float32 device tensor -> same shape."""
        x = x.contiguous()
        out = torch.empty_like(x)
        self._check(lib().feast_nh_net_forward(self.h, _ptr(x), _ptr(out), x.shape[0]), "forward")
        return out

    def train_step(self, x, target, lr, want_grad=False):
        """One step on the MSE of the first target.shape[-1] channels; returns
        (loss, gradient or None)."""
        x, target = x.contiguous(), target.contiguous()
        loss = C.c_double()
        grad = torch.empty(self.layers * NET_LAYER_PARAMS, dtype=torch.float32, device=self.device) \
            if want_grad else None
        self._check(lib().feast_nh_net_train_step(self.h, _ptr(x), _ptr(target), target.shape[-1], x.shape[0],
                                                  float(lr), C.byref(loss), _ptr(grad)), "train_step")
        return loss.value, grad

    def backward(self, gout, lr, want_grad=False):
        """Backward from d loss / d out of the last forward, optional Adam step."""
        gout = gout.contiguous()
        grad = torch.empty(self.layers * NET_LAYER_PARAMS, dtype=torch.float32, device=self.device) \
            if want_grad else None
        self._check(lib().feast_nh_net_backward(self.h, _ptr(gout), gout.shape[0], float(lr), _ptr(grad)), "backward")
        return grad

    def close(self):
        if getattr(self, "h", None):
            lib().feast_nh_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def train_operator_loss(net, ctx, Xin, T, N, steps, lr, batch, generator=None):
    """Training loop of the learned preconditioner on exact-solve pairs (the
    arithmetic runs in the library: forward, operator-norm loss, backward,
    Adam).  Batches of `batch` whole node groups (all ne systems of a column
    are kept together, as feast_nh_operator_loss pairs image s with node
    s // m).  Returns the losses."""
    ne = ctx.ne
    m = Xin.shape[0] // ne
    losses = []
    cols = max(1, batch // ne)
    for _ in range(steps):
        c = torch.randperm(m, generator=generator, device="cpu")[:cols]
        idx = (torch.arange(ne)[:, None] * m + c[None, :]).reshape(-1).to(Xin.device)
        out = net.forward(Xin[idx])
        loss, g = _batch_operator_loss(ctx, out, T[idx], N, ne, cols)
        net.backward(g, lr)
        losses.append(loss)
    return losses


def _batch_operator_loss(ctx, out, T, N, ne, cols):
    # the selected images are node-major (j * cols + c): the same layout the
    # library uses for ne nodes x cols columns
    out, T = out.contiguous(), T.contiguous()
    g = torch.empty_like(out)
    loss = C.c_double()
    st = lib().feast_nh_operator_loss(ctx.h, _ptr(out), _ptr(T), cols, int(N), 0, _ptr(g), C.byref(loss))
    ctx._check(st, "feast_nh_operator_loss")
    return loss.value, g
