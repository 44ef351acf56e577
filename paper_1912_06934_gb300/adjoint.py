"""Differentiable MsRSB solve (adjoint method) and a differentiable TPFA
forward model, for gradients of objectives of the pressure with respect to
log-permeability.

MsrsbSolve is a torch.autograd.Function for x = A^-1 b with A given by its
values on a fixed sparse pattern. Its backward pass solves the adjoint system
A^T lambda = dJ/dx with the MsRSB-preconditioned Krylov solver, set up afresh
on A^T (msrsb_transpose_values gives A^T's values in A's symmetric pattern;
the basis is recomputed, not stored), and returns dJ/db = lambda and
dJ/dA = -lambda x^T on the pattern (msrsb_pattern_outer). Every step of the
solves and of the gradient runs in the library's kernels; torch only chains
them with the forward model.

MsrsbMpfaSolve is the same for the MPFA-O Darcy model of the 27-point
workloads (3D unit cells, K_c = exp(theta_c) K_hat_c, no-flow outer faces,
bottom-hole-pressure wells): p = A(theta)^-1 b(theta), assembled on the GPU
(msrsb_mpfa_assemble), with dJ/dtheta = -lambda^T (dA/dtheta) p + lambda^T
(db/dtheta) from the interaction regions' local systems (msrsb_mpfa_gradient).

tpfa_darcy builds A(log k) and b(log k) of a two-point flux discretisation on
a Cartesian grid of unit cells (isotropic k, harmonic-mean face
transmissibilities, p = 1 on the x = 0 face and p = 0 on the x = nx face, no
flow elsewhere) with torch operations, so that autograd carries dJ/dA and
dJ/db back to dJ/d log k.
"""
import numpy as np
import torch

from .msrsb import (Mat, msrsb_mpfa_assemble, msrsb_mpfa_gradient, msrsb_pattern_outer, msrsb_setup, msrsb_spmv,
                    msrsb_transpose_values)


def _refined_solve(h, A, b, rtol, maxit, refine):
    """x = A^-1 b by the MsRSB-preconditioned solve, then `refine` steps of
    iterative refinement (r = b - A x in FP64, x += A^-1 r): each step
    carries the solve's relative tolerance to the correction, past what one
    Krylov solve attains on ill-conditioned well problems."""
    x = h.solve(b, rtol=rtol, maxit=maxit)["x"]
    for _ in range(refine):
        r = b - msrsb_spmv(A, x)
        if float(torch.linalg.vector_norm(r)) == 0.0:
            break
        x = x + h.solve(r, rtol=rtol, maxit=maxit)["x"]
    return x


class MsrsbSolve(torch.autograd.Function):
    """x = A^-1 b. Inputs: vals (CUDA FP64, A's values on the pattern), b
    (CUDA FP64), pattern = (rowptr, colidx, bdim, grid), o (msrsb_opts),
    rtol, maxit."""

    @staticmethod
    def forward(ctx, vals, b, pattern, o, rtol, maxit):
        rowptr, colidx, bdim, g = pattern
        A = Mat(rowptr, colidx, vals.detach().contiguous(), bdim)
        h = msrsb_setup(A, g, o)
        x = h.solve(b.detach().contiguous(), rtol=rtol, maxit=maxit)["x"]
        h.destroy()
        ctx.save_for_backward(vals, x)
        ctx.meta = (pattern, o, rtol, maxit)
        return x

    @staticmethod
    def backward(ctx, gx):
        vals, x = ctx.saved_tensors
        (rowptr, colidx, bdim, g), o, rtol, maxit = ctx.meta
        A = Mat(rowptr, colidx, vals.detach().contiguous(), bdim)
        At = Mat(rowptr, colidx, msrsb_transpose_values(A), bdim)
        h = msrsb_setup(At, g, o)
        lam = h.solve(gx.contiguous(), rtol=rtol, maxit=maxit)["x"]
        h.destroy()
        gvals = msrsb_pattern_outer(A, -1.0, lam, x) if ctx.needs_input_grad[0] else None
        gb = lam if ctx.needs_input_grad[1] else None
        return gvals, gb, None, None, None, None


class MsrsbMpfaSolve(torch.autograd.Function):
    """p = A(theta)^-1 b(theta) for the MPFA-O model. Inputs: theta (CUDA
    FP64, n), model = (grid, K_hat (n, 3, 3) CUDA FP64, wells [(cell, p_w)],
    rowptr, colidx of the 27-point pattern), o (msrsb_opts), rtol, maxit,
    refine (iterative-refinement steps after each solve)."""

    @staticmethod
    def forward(ctx, theta, model, o, rtol, maxit, refine):
        g, K_hat, wells, rowptr, colidx = model
        th = theta.detach().contiguous()
        val, b = msrsb_mpfa_assemble(g, K_hat, th, wells, rowptr, colidx)
        A = Mat(rowptr, colidx, val)
        h = msrsb_setup(A, g, o)
        p = _refined_solve(h, A, b, rtol, maxit, refine)
        h.destroy()
        ctx.save_for_backward(th, val, p)
        ctx.meta = (model, o, rtol, maxit, refine)
        return p

    @staticmethod
    def backward(ctx, gp):
        th, val, p = ctx.saved_tensors
        (g, K_hat, wells, rowptr, colidx), o, rtol, maxit, refine = ctx.meta
        A = Mat(rowptr, colidx, val)
        At = Mat(rowptr, colidx, msrsb_transpose_values(A))
        h = msrsb_setup(At, g, o)
        lam = _refined_solve(h, At, gp.contiguous(), rtol, maxit, refine)
        h.destroy()
        return msrsb_mpfa_gradient(g, K_hat, th, wells, lam, p), None, None, None, None, None


def msrsb_mpfa_solve_diff(theta, model, o, rtol=1e-10, maxit=500, refine=0):
    """Differentiable p = A(theta)^-1 b(theta) of the MPFA-O model (see
    MsrsbMpfaSolve)."""
    return MsrsbMpfaSolve.apply(theta, model, o, rtol, maxit, refine)


def msrsb_solve_diff(vals, b, pattern, o, rtol=1e-10, maxit=500):
    """Differentiable x = A(vals)^-1 b (see MsrsbSolve)."""
    return MsrsbSolve.apply(vals, b, pattern, o, rtol, maxit)


def tpfa_pattern(dims, device="cuda"):
    """CSR pattern (rowptr, colidx int32, columns ascending) of the 5- or
    7-point stencil on a grid of dims (x fastest), and for every entry its
    kind: -1 for the diagonal, else the index of the face it stands for."""
    d = len(dims)
    n = int(np.prod(dims))
    idx = np.arange(n).reshape(dims[::-1])  # [z][y][x] (x fastest)
    faces_l, faces_r = [], []
    for a in range(d):
        ax = d - 1 - a  # numpy axis of grid axis a
        lo = np.take(idx, np.arange(dims[a] - 1), axis=ax).ravel()
        hi = np.take(idx, np.arange(1, dims[a]), axis=ax).ravel()
        faces_l.append(lo)
        faces_r.append(hi)
    fl = np.concatenate(faces_l)
    fr = np.concatenate(faces_r)
    nf = len(fl)
    rows = np.concatenate([np.arange(n), fl, fr])
    cols = np.concatenate([np.arange(n), fr, fl])
    kind = np.concatenate([-np.ones(n, dtype=np.int64), np.arange(nf), np.arange(nf)])
    order = np.lexsort((cols, rows))
    rows, cols, kind = rows[order], cols[order], kind[order]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    t = lambda a, dt: torch.as_tensor(a.astype(dt), device=device)  # noqa: E731
    return dict(n=n, rowptr=t(rowptr, np.int32), colidx=t(cols, np.int32), rows=t(rows, np.int64),
                kind=t(kind, np.int64), fl=t(fl, np.int64), fr=t(fr, np.int64),
                west=t(np.take(idx, [0], axis=d - 1).ravel(), np.int64),
                east=t(np.take(idx, [dims[0] - 1], axis=d - 1).ravel(), np.int64))


def tpfa_darcy(logk, pat):
    """(vals, b) of the TPFA system for cell log-permeabilities logk (CUDA
    FP64, length n): face transmissibility 2 k_L k_R / (k_L + k_R) between
    unit cells, Dirichlet faces with transmissibility 2 k (half a cell);
    differentiable in logk."""
    k = torch.exp(logk)
    kl, kr = k[pat["fl"]], k[pat["fr"]]
    T = 2.0 * kl * kr / (kl + kr)
    n = pat["n"]
    diag = torch.zeros(n, dtype=k.dtype, device=k.device)
    diag = diag.index_add(0, pat["fl"], T).index_add(0, pat["fr"], T)
    Tw, Te = 2.0 * k[pat["west"]], 2.0 * k[pat["east"]]
    diag = diag.index_add(0, pat["west"], Tw).index_add(0, pat["east"], Te)
    b = torch.zeros(n, dtype=k.dtype, device=k.device).index_add(0, pat["west"], Tw)
    kind = pat["kind"]
    off = -T[kind.clamp(min=0)]
    vals = torch.where(kind < 0, diag[pat["rows"]], off)
    return vals, b
