"""Thin ctypes binding of libmsrsb.so (include/msrsb.h): argument marshalling only.

Every entry point of the C ABI has a function of the same name here. Device
arrays are torch CUDA tensors; PyTorch provides memory and the current stream.
There is no CPU path: if the library is missing, calls raise.
"""
import ctypes
import os

import torch

from . import _build

_LIB = None

MSRSB_OK, MSRSB_EINVAL, MSRSB_ESHAPE, MSRSB_ECUDA, MSRSB_ENOMEM = 0, 1, 2, 3, 4
MSRSB_EBREAKDOWN, MSRSB_ENOCONV, MSRSB_ETIMEOUT, MSRSB_ENAN = 5, 6, 7, 8
MSRSB_F64, MSRSB_F32 = 0, 1
MSRSB_SMOOTH_NONE, MSRSB_SMOOTH_ILU0, MSRSB_SMOOTH_GS, MSRSB_SMOOTH_L1JAC, MSRSB_SMOOTH_IC0 = 0, 1, 2, 3, 4
MSRSB_GMRES, MSRSB_PCG, MSRSB_RICHARDSON = 0, 1, 2
MSRSB_RESTRICT_GALERKIN, MSRSB_RESTRICT_FV = 0, 1
MSRSB_ORDER_LINES, MSRSB_ORDER_PARITY = 0, 1
MSRSB_TUNE_AUTO, MSRSB_TUNE_SMOOTH = -1, 0

EXPORTS = ["msrsb_partition_size", "msrsb_partition", "msrsb_filter", "msrsb_build_basis", "msrsb_coarse_op",
           "msrsb_setup", "msrsb_apply", "msrsb_solve", "msrsb_get_setup", "msrsb_get_info", "msrsb_destroy",
           "msrsb_solve_host", "msrsb_profile", "msrsb_profile_read", "msrsb_wait_selftest", "msrsb_build_basis_noalloc",
           "msrsb_solve_ensemble", "msrsb_transpose_values", "msrsb_pattern_outer", "msrsb_fma_rate", "msrsb_mpfa_assemble", "msrsb_mpfa_gradient", "msrsb_spmv", "msrsb_solve_multi", "msrsb_tune_mode", "msrsb_tune_reset",
           "msrsb_tune_table", "msrsb_last_error"]


class MsrsbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("msrsb status %d: %s" % (status, msg))
        self.status = status


class c_mat(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("nnz", ctypes.c_int32), ("bdim", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class c_grid(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("dim", "nx", "ny", "nz", "hx", "hy", "hz", "centering", "ncomp")]


class c_basis_opts(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("tol", ctypes.c_double), ("n_it", ctypes.c_int32),
                ("max_iter", ctypes.c_int32)]


class c_opts(ctypes.Structure):
    _fields_ = [("basis", c_basis_opts), ("smoother", ctypes.c_int32), ("pre", ctypes.c_int32),
                ("post", ctypes.c_int32), ("krylov", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("no_coarse", ctypes.c_int32), ("restriction", ctypes.c_int32),
                ("ordering", ctypes.c_int32)]


class c_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("bdim", ctypes.c_int32), ("nc", ctypes.c_int32), ("W", ctypes.c_int32),
                ("basis_iters", ctypes.c_int32), ("basis_e_it", ctypes.c_double),
                ("n_zero_diag", ctypes.c_int32), ("ncolours", ctypes.c_int32), ("phase_ms", ctypes.c_double * 7)]


class c_problem(ctypes.Structure):
    _fields_ = [("A", ctypes.POINTER(c_mat)), ("g", ctypes.POINTER(c_grid)), ("b", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("nrhs", ctypes.c_int32), ("iters_h", ctypes.POINTER(ctypes.c_int32)),
                ("relres_h", ctypes.POINTER(ctypes.c_double)), ("status", ctypes.c_int)]


def lib_path():
    return _build.LIB


def load(path=None):
    """Load libmsrsb.so (no device work). Raises if it has not been built."""
    global _LIB
    if _LIB is None:
        p = path or lib_path()
        if not os.path.exists(p):
            raise RuntimeError("libmsrsb.so is not built (expected at %s); run __graft_entry__.build()" % p)
        lib = ctypes.CDLL(p)
        lib.msrsb_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "msrsb_last_error":
                getattr(lib, name).restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _check(st):
    if st != MSRSB_OK:
        raise MsrsbError(st, load().msrsb_last_error().decode())
    return st


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Mat:
    """FP64 fine operator on the device: CSR (bdim 1) or 3x3 block CSR (bdim 3)."""

    def __init__(self, rowptr, colidx, val, bdim=1):
        self.rowptr, self.colidx, self.val, self.bdim = rowptr, colidx, val, bdim
        self.nrows = rowptr.numel() - 1
        self.nnz = colidx.numel()
        assert rowptr.dtype == torch.int32 and colidx.dtype == torch.int32 and val.dtype == torch.float64
        assert val.numel() == self.nnz * bdim * bdim

    @classmethod
    def from_host(cls, indptr, indices, data, bdim=1, device="cuda"):
        import numpy as np
        return cls(torch.as_tensor(np.ascontiguousarray(indptr, dtype=np.int32), device=device),
                   torch.as_tensor(np.ascontiguousarray(indices, dtype=np.int32), device=device),
                   torch.as_tensor(np.ascontiguousarray(data, dtype=np.float64).reshape(-1), device=device), bdim)

    def c(self):
        return c_mat(self.nrows, self.nnz, self.bdim, self.rowptr.data_ptr(), self.colidx.data_ptr(),
                     self.val.data_ptr())


def grid(dims, H, centering=0, ncomp=1):
    d = len(dims)
    nz = dims[2] if d == 3 else 1
    hz = H[2] if d == 3 else 1
    return c_grid(d, dims[0], dims[1], nz, H[0], H[1], hz, centering, ncomp)


def basis_opts(omega=2.0 / 3.0, tol=1e-3, n_it=10, max_iter=100):
    return c_basis_opts(omega, tol, n_it, max_iter)


def opts(omega=2.0 / 3.0, tol=1e-3, n_it=10, max_iter=100, smoother=MSRSB_SMOOTH_ILU0, pre=0, post=1,
         krylov=MSRSB_GMRES, restart=200, prec=MSRSB_F64, no_coarse=0, restriction=MSRSB_RESTRICT_GALERKIN,
         ordering=MSRSB_ORDER_LINES):
    return c_opts(basis_opts(omega, tol, n_it, max_iter), smoother, pre, post, krylov, restart, prec, no_coarse,
                  restriction, ordering)


def _pdtype(prec):
    return torch.float64 if prec == MSRSB_F64 else torch.float32


def msrsb_partition_size(g):
    n, nc, W = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().msrsb_partition_size(ctypes.byref(g), ctypes.byref(n), ctypes.byref(nc), ctypes.byref(W)))
    return n.value, nc.value, W.value


def msrsb_partition(g, stream=None, device="cuda"):
    n, nc, W = msrsb_partition_size(g)
    part = torch.empty(n, dtype=torch.int32, device=device)
    cnode = torch.empty(nc, dtype=torch.int32, device=device)
    p_ids = torch.empty(n * W, dtype=torch.int32, device=device)
    skel = torch.empty(n, dtype=torch.uint8, device=device)
    _check(load().msrsb_partition(ctypes.byref(g), _ptr(part), _ptr(cnode), _ptr(p_ids), _ptr(skel),
                                  _stream(stream)))
    return part, cnode, p_ids.view(n, W), skel


def msrsb_filter(A, comp=0, stream=None):
    ahat = torch.empty(A.nnz, dtype=torch.float64, device=A.val.device)
    nz = ctypes.c_int32()
    m = A.c()
    _check(load().msrsb_filter(ctypes.byref(m), ctypes.c_int32(comp), _ptr(ahat), ctypes.byref(nz), _stream(stream)))
    return ahat, nz.value


def msrsb_build_basis(Ahat, p_ids, skel, W, bopts, prec, p_val, stream=None):
    """Alg. 1 in place on p_val ([n][W], dtype matching prec). Returns (iters, e_it)."""
    assert p_val.dtype == _pdtype(prec) and p_val.is_contiguous()
    it, e = ctypes.c_int32(), ctypes.c_double()
    m = Ahat.c()
    _check(load().msrsb_build_basis(ctypes.byref(m), _ptr(p_ids), _ptr(skel), ctypes.c_int32(W), ctypes.byref(bopts),
                                    ctypes.c_int32(prec), _ptr(p_val), ctypes.byref(it), ctypes.byref(e),
                                    _stream(stream)))
    return it.value, e.value


def msrsb_build_basis_noalloc(Ahat, p_ids, skel, W, bopts, prec, p_val, stream=None):
    """Allocation-free variant of msrsb_build_basis (static device scratch;
    see include/msrsb.h for its limits). Returns (iters, e_it)."""
    assert p_val.dtype == _pdtype(prec) and p_val.is_contiguous()
    it, e = ctypes.c_int32(), ctypes.c_double()
    m = Ahat.c()
    _check(load().msrsb_build_basis_noalloc(ctypes.byref(m), _ptr(p_ids), _ptr(skel), ctypes.c_int32(W),
                                            ctypes.byref(bopts), ctypes.c_int32(prec), _ptr(p_val), ctypes.byref(it),
                                            ctypes.byref(e), _stream(stream)))
    return it.value, e.value


def msrsb_coarse_op(A, g, p_ids, p_val, prec, stream=None):
    """A_c = P^T A P as block CSR device tensors (rowptr[nc+1], colidx[nnzb],
    val[nnzb, bdim, bdim])."""
    n, nc, W = msrsb_partition_size(g)
    m = A.c()
    nnzb = ctypes.c_int32()
    _check(load().msrsb_coarse_op(ctypes.byref(m), ctypes.byref(g), None, None, ctypes.c_int32(prec), None, None,
                                  None, ctypes.byref(nnzb), _stream(stream)))
    dev = A.val.device
    rowptr = torch.empty(nc + 1, dtype=torch.int32, device=dev)
    colidx = torch.empty(nnzb.value, dtype=torch.int32, device=dev)
    val = torch.empty((nnzb.value, A.bdim, A.bdim), dtype=torch.float64, device=dev)
    _check(load().msrsb_coarse_op(ctypes.byref(m), ctypes.byref(g), _ptr(p_ids), _ptr(p_val), ctypes.c_int32(prec),
                                  _ptr(rowptr), _ptr(colidx), _ptr(val), ctypes.byref(nnzb), _stream(stream)))
    return rowptr, colidx, val


class Handle:
    """Owns an msrsb_handle*. Keeps a reference to A's tensors (the library
    holds non-owning pointers to them until destroy)."""

    def __init__(self, A, g, o, p_init=None, stream=None):
        self.A, self.grid, self.opts = A, g, o
        self._h = ctypes.c_void_p()
        m = A.c()
        _check(load().msrsb_setup(ctypes.byref(m), ctypes.byref(g), ctypes.byref(o), _ptr(p_init),
                                  ctypes.byref(self._h), _stream(stream)))

    def info(self):
        inf = c_info()
        _check(load().msrsb_get_info(self._h, ctypes.byref(inf)))
        out = {k: getattr(inf, k) for k, _ in c_info._fields_}
        out["phase_ms"] = list(inf.phase_ms)
        return out

    def apply(self, v, z=None, stream=None):
        z = torch.empty_like(v) if z is None else z
        _check(load().msrsb_apply(self._h, _ptr(v), _ptr(z), _stream(stream)))
        return z

    def solve(self, b, x=None, rtol=1e-8, maxit=200, hist=False, stream=None, raise_on_noconv=True):
        x = torch.zeros_like(b) if x is None else x
        it, rr = ctypes.c_int32(), ctypes.c_double()
        hbuf = (ctypes.c_double * (maxit + 2))() if hist else None
        st = load().msrsb_solve(self._h, _ptr(b), _ptr(x), ctypes.c_double(rtol), ctypes.c_int32(maxit),
                                ctypes.byref(it), ctypes.byref(rr), hbuf, _stream(stream))
        if st != MSRSB_OK and (st != MSRSB_ENOCONV or raise_on_noconv):
            _check(st)
        out = dict(x=x, iters=it.value, relres=rr.value, status=st)
        if hist:
            out["hist"] = list(hbuf)[: it.value + 1]
        return out

    def solve_multi(self, B, X=None, rtol=1e-8, maxit=200, stream=None):
        """msrsb_solve_multi: B (nrhs, n*bdim) CUDA FP64, one right-hand side
        per row; returns dict(x=(nrhs, n*bdim), iters=[...], relres=[...])."""
        B = B.contiguous()
        X = torch.zeros_like(B) if X is None else X
        k = B.shape[0]
        its = (ctypes.c_int32 * max(k, 1))()
        rr = (ctypes.c_double * max(k, 1))()
        _check(load().msrsb_solve_multi(self._h, ctypes.c_int32(k), _ptr(B), _ptr(X), ctypes.c_double(rtol),
                                        ctypes.c_int32(maxit), its, rr, _stream(stream)))
        return dict(x=X, iters=list(its)[:k], relres=list(rr)[:k])

    def get_setup(self, stream=None):
        inf = self.info()
        n, W, bd, nc = inf["n"], inf["W"], inf["bdim"], inf["nc"]
        dev = self.A.val.device
        p_ids = torch.empty((n, W), dtype=torch.int32, device=dev)
        p_val = torch.empty((bd, n, W), dtype=_pdtype(self.opts.prec), device=dev)
        Ac = torch.empty((nc * bd, nc * bd), dtype=torch.float64, device=dev)
        _check(load().msrsb_get_setup(self._h, _ptr(p_ids), _ptr(p_val), _ptr(Ac), _stream(stream)))
        return p_ids, p_val, Ac

    def destroy(self):
        if self._h:
            _check(load().msrsb_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def msrsb_setup(A, g, o, p_init=None, stream=None):
    return Handle(A, g, o, p_init, stream)


def msrsb_apply(h, v, z=None, stream=None):
    return h.apply(v, z, stream)


def msrsb_solve(h, b, x=None, rtol=1e-8, maxit=200, hist=False, stream=None):
    return h.solve(b, x, rtol, maxit, hist, stream)


def msrsb_get_setup(h, stream=None):
    return h.get_setup(stream)


def msrsb_get_info(h):
    return h.info()


def msrsb_destroy(h):
    h.destroy()


def msrsb_profile(enable):
    _check(load().msrsb_profile(ctypes.c_int32(1 if enable else 0)))


def msrsb_wait_selftest(limit_ms=20.0, stream=None):
    """Run the bounded-wait self-test (see include/msrsb.h); returns the raw
    status, MSRSB_ETIMEOUT when the wait expired and reported it."""
    L = load()
    L.msrsb_wait_selftest.restype = ctypes.c_int
    L.msrsb_wait_selftest.argtypes = [ctypes.c_double, ctypes.c_void_p]
    return int(L.msrsb_wait_selftest(float(limit_ms), _stream(stream)))


def msrsb_fma_rate(prec, blocks_per_sm=8, stream=None):
    """(FMAs per second, ms of the best launch) of the arithmetic-rate probe."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().msrsb_fma_rate(ctypes.c_int32(prec), ctypes.c_int32(blocks_per_sm), ctypes.byref(r),
                                 ctypes.byref(ms), _stream(stream)))
    return r.value, ms.value


class c_tune_entry(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("kernel", "device", "value_bytes", "W", "n_log2", "width_log2",
                                              "variant", "lanes", "threads", "ahead", "capped", "n_variants")] + \
               [("us", ctypes.c_float * 8)]


def msrsb_tune_mode(mode):
    """MSRSB_TUNE_AUTO (time the launch shapes of a new size class) or a
    forced shape index 0..5 (see include/msrsb.h)."""
    _check(load().msrsb_tune_mode(ctypes.c_int32(mode)))


def msrsb_tune_reset():
    _check(load().msrsb_tune_reset())


def msrsb_tune_table():
    """The autotuner's decisions: one dict per size class."""
    L = load()
    cnt = ctypes.c_int32()
    _check(L.msrsb_tune_table(None, ctypes.c_int32(0), ctypes.byref(cnt)))
    n = cnt.value
    arr = (c_tune_entry * max(n, 1))()
    _check(L.msrsb_tune_table(arr, ctypes.c_int32(n), ctypes.byref(cnt)))
    out = []
    for e in arr[:min(n, cnt.value)]:
        d = {k: getattr(e, k) for k, _ in c_tune_entry._fields_ if k != "us"}
        d["us"] = [round(float(v), 3) for v in e.us[:e.n_variants]]
        out.append(d)
    return out


def msrsb_profile_read():
    """(kernel launches since reset, smoothing launches timed, their total ms)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(load().msrsb_profile_read(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def msrsb_solve_host(indptr, indices, data, bdim, g, o, b, x, rtol=1e-8, maxit=200, stream=None):
    """End-to-end call with host arrays (numpy or pinned torch CPU tensors):
    copies in, set-up, solve, copies x out. Returns (iters, relres)."""
    import numpy as np
    ip = np.ascontiguousarray(indptr, dtype=np.int32)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    dv = np.ascontiguousarray(data, dtype=np.float64)
    m = c_mat(len(ip) - 1, len(ix), bdim, ip.ctypes.data, ix.ctypes.data, dv.ctypes.data)
    it, rr = ctypes.c_int32(), ctypes.c_double()
    bp = ctypes.c_void_p(b.data_ptr()) if isinstance(b, torch.Tensor) else ctypes.c_void_p(b.ctypes.data)
    xp = ctypes.c_void_p(x.data_ptr()) if isinstance(x, torch.Tensor) else ctypes.c_void_p(x.ctypes.data)
    _check(load().msrsb_solve_host(ctypes.byref(m), ctypes.byref(g), ctypes.byref(o), bp, xp, ctypes.c_double(rtol),
                                   ctypes.c_int32(maxit), ctypes.byref(it), ctypes.byref(rr), _stream(stream)))
    return it.value, rr.value


def msrsb_solve_host_ptrs(indptr, indices, data, bdim, g, o, b, x, rtol=1e-8, maxit=200, stream=None):
    """msrsb_solve_host on torch CPU tensors (pinned for asynchronous copies);
    x receives the solution. Returns (iters, relres)."""
    for t in (indptr, indices, data, b, x):
        assert not t.is_cuda and t.is_contiguous()
    m = c_mat(indptr.numel() - 1, indices.numel(), bdim, indptr.data_ptr(), indices.data_ptr(), data.data_ptr())
    it, rr = ctypes.c_int32(), ctypes.c_double()
    _check(load().msrsb_solve_host(ctypes.byref(m), ctypes.byref(g), ctypes.byref(o), _ptr(b), _ptr(x),
                                   ctypes.c_double(rtol), ctypes.c_int32(maxit), ctypes.byref(it), ctypes.byref(rr),
                                   _stream(stream)))
    return it.value, rr.value


def msrsb_solve_ensemble(problems, o, rtol=1e-8, maxit=200, concurrency=4):
    """problems: list of (Mat, grid, B, X) with B, X CUDA FP64 tensors of shape
    (nrhs, n*bdim) (X: initial guesses, overwritten by the solutions). Returns
    (iters, relres, status) per problem. The calls run on streams of the
    library's own, so the current stream is synchronised first."""
    torch.cuda.current_stream().synchronize()
    keep, arr = [], (c_problem * len(problems))()
    for i, (A, g, B, X) in enumerate(problems):
        assert B.dtype == torch.float64 and X.dtype == torch.float64 and B.is_contiguous() and X.is_contiguous()
        nrhs = B.shape[0]
        m = A.c()
        its = (ctypes.c_int32 * max(nrhs, 1))()
        rr = (ctypes.c_double * max(nrhs, 1))()
        keep.append((m, g, its, rr, nrhs))
        arr[i] = c_problem(ctypes.pointer(m), ctypes.pointer(g), B.data_ptr(), X.data_ptr(), nrhs,
                           ctypes.cast(its, ctypes.POINTER(ctypes.c_int32)),
                           ctypes.cast(rr, ctypes.POINTER(ctypes.c_double)), 0)
    st = load().msrsb_solve_ensemble(ctypes.c_int32(len(problems)), arr, ctypes.byref(o), ctypes.c_double(rtol),
                                     ctypes.c_int32(maxit), ctypes.c_int32(concurrency))
    out = [(list(k[2])[:k[4]], list(k[3])[:k[4]], arr[i].status) for i, k in enumerate(keep)]
    _check(st)
    return out


def _wells(wells):
    import numpy as np
    cells = np.ascontiguousarray([w[0] for w in wells], dtype=np.int32)
    pw = np.ascontiguousarray([w[1] for w in wells], dtype=np.float64)
    return len(wells), cells, pw


def msrsb_mpfa_assemble(g, K_hat, theta, wells, rowptr, colidx, stream=None):
    """MPFA-O values (in the given 27-point CSR pattern) and b for cell
    log-permeabilities theta; K_hat (n, 3, 3) and theta device FP64 tensors;
    wells a list of (cell, pressure). Returns (val, b)."""
    nw, wc, wp = _wells(wells)
    val = torch.empty(colidx.numel(), dtype=torch.float64, device=theta.device)
    b = torch.empty(theta.numel(), dtype=torch.float64, device=theta.device)
    _check(load().msrsb_mpfa_assemble(ctypes.byref(g), _ptr(K_hat.contiguous()), _ptr(theta.contiguous()),
                                      ctypes.c_int32(nw), ctypes.c_void_p(wc.ctypes.data),
                                      ctypes.c_void_p(wp.ctypes.data), _ptr(rowptr), _ptr(colidx), _ptr(val), _ptr(b),
                                      _stream(stream)))
    return val, b


def msrsb_mpfa_gradient(g, K_hat, theta, wells, lam, p, stream=None):
    """dJ/dtheta = -lambda^T dA/dtheta p + lambda^T db/dtheta (device tensor)."""
    nw, wc, wp = _wells(wells)
    grad = torch.empty_like(theta)
    _check(load().msrsb_mpfa_gradient(ctypes.byref(g), _ptr(K_hat.contiguous()), _ptr(theta.contiguous()),
                                      ctypes.c_int32(nw), ctypes.c_void_p(wc.ctypes.data),
                                      ctypes.c_void_p(wp.ctypes.data), _ptr(lam.contiguous()), _ptr(p.contiguous()),
                                      _ptr(grad), _stream(stream)))
    return grad


def msrsb_spmv(A, x, y=None, stream=None):
    """y = A x (device FP64 vectors)."""
    y = torch.empty_like(x) if y is None else y
    _check(load().msrsb_spmv(ctypes.byref(A.c()), _ptr(x), _ptr(y), _stream(stream)))
    return y


def msrsb_transpose_values(A, stream=None):
    """Values of A^T in A's (structurally symmetric) pattern, as a new tensor."""
    out = torch.empty_like(A.val)
    _check(load().msrsb_transpose_values(ctypes.byref(A.c()), _ptr(out), _stream(stream)))
    return out


def msrsb_pattern_outer(A, alpha, lam, x, stream=None):
    """alpha * lam x^T on A's pattern (same layout as A.val)."""
    out = torch.empty_like(A.val)
    _check(load().msrsb_pattern_outer(ctypes.byref(A.c()), ctypes.c_double(alpha), _ptr(lam), _ptr(x), _ptr(out),
                                      _stream(stream)))
    return out
