"""FP64 CPU oracle of the enhanced MsRSB two-level preconditioner.

TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the CPU-baseline leg
of bench.py may import this module; the library's product path never does.
It shares no code with the CUDA path.

Every function restates a step of Bosma, Klevtsov, Moyner, Castelletto,
"Enhanced multiscale restriction-smoothed basis (MsRSB) preconditioning with
applications to porous media flow and geomechanics" (arXiv 1912.06934) in plain
numpy/scipy, slowly and in the paper's order; the passage is cited in each
docstring. Where the paper is silent the documented reading is given inline.

Matrices are scipy CSR (float64, sorted column indices). The prolongation P is
kept on its fixed support pattern: ``pat`` is a CSR pattern (n rows, nc
columns, sorted coarse ids per row) and ``vals`` the values on it.
"""
import ctypes
import os
import subprocess

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------
# primal partition, coarse nodes, support regions (Sec. 2.1, Fig. 1; the
# initial basis is the indicator of the primal block, Sec. 2.1)
# ----------------------------------------------------------------------------


def coarse_axis(n, H, centering):
    """One grid axis: coarse-node coordinates c_I and the block of each point.

    Cell-centred (FV): block I holds cells [I*H, min((I+1)*H, n)); its coarse
    node is the lower-middle cell of the block (the paper only asks for a
    representative fine cell). Vertex-centred (FE): coarse nodes sit on nodes
    0, H, 2H, ... (the last one clamped to n-1) and each node belongs to the
    block of its nearest coarse node, ties going to the lower one.
    Returns (c, block) with c sorted ascending.
    """
    x = np.arange(n)
    if centering == 0:
        nb = -(-n // H)
        c = np.array([I * H + (min((I + 1) * H, n) - I * H - 1) // 2 for I in range(nb)])
        block = x // H
    else:
        nb = -(-(n - 1) // H) + 1
        c = np.array([min(I * H, n - 1) for I in range(nb)])
        dist = np.abs(x[:, None] - c[None, :])
        block = np.argmin(dist, axis=1)  # argmin takes the first (lower) on ties
    return c, block


def axis_supports(n, c):
    """Support of coarse node I along one axis: the open interval
    (c_{I-1}, c_{I+1}), reaching the domain edge where there is no neighbour.
    A point exactly on c_J (J != I) bounds I's support (support boundary); the
    points with coordinate c_I are I's support edge. Returns a boolean
    (n, nb) matrix S[x, I] = x in supp_I."""
    nb = len(c)
    S = np.zeros((n, nb), dtype=bool)
    for I in range(nb):
        lo = c[I - 1] if I > 0 else -1
        hi = c[I + 1] if I + 1 < nb else n
        S[lo + 1:hi, I] = True
    return S


def partition(dims, H, centering):
    """Primal partition and the support pattern of P on a Cartesian grid.

    Returns dict with
      part[n]     primal block (flat coarse id) of every fine point,
      cnode[nc]   flat fine index of every coarse node,
      pat         CSR pattern (n x nc): coarse ids whose support holds the row,
      skel[n]     True where the point lies on any coarse-node line, i.e. on a
                  support edge of some basis (and a boundary of another).
    Flat orders have x fastest, for fine points and coarse ids alike.
    """
    d = len(dims)
    axes = [coarse_axis(dims[a], H[a], centering) for a in range(d)]
    nbs = [len(c) for c, _ in axes]
    n = int(np.prod(dims))
    nc = int(np.prod(nbs))
    coords = np.indices(dims).reshape(d, -1, order="F")
    part = np.zeros(n, dtype=np.int64)
    stride = 1
    for a in range(d):
        part += axes[a][1][coords[a]] * stride
        stride *= nbs[a]
    cc = np.indices(nbs).reshape(d, -1, order="F")
    cnode = np.zeros(nc, dtype=np.int64)
    stride = 1
    for a in range(d):
        cnode += axes[a][0][cc[a]] * stride
        stride *= dims[a]
    supp = [axis_supports(dims[a], axes[a][0]) for a in range(d)]
    # row pattern = tensor product of the per-axis memberships
    rows, cols = [], []
    per_axis = [[np.flatnonzero(supp[a][x]) for x in range(dims[a])] for a in range(d)]
    skel = np.zeros(n, dtype=bool)
    for a in range(d):
        skel |= np.isin(coords[a], axes[a][0])
    for i in range(n):
        ids = np.zeros(1, dtype=np.int64)
        stride = 1
        for a in range(d):
            ids = (ids[:, None] + per_axis[a][coords[a][i]][None, :] * stride).ravel()
            stride *= nbs[a]
        ids.sort()
        rows.append(np.full(len(ids), i))
        cols.append(ids)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    pat = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, nc))
    pat.sort_indices()
    return dict(part=part, cnode=cnode, pat=pat, skel=skel, nb=tuple(nbs), nc=nc)


def indicator(part, pat):
    """Initial basis: P0_iJ = 1 if fine point i lies in primal block J (Sec. 2.1)."""
    rows = np.repeat(np.arange(pat.shape[0]), np.diff(pat.indptr))
    return (pat.indices == part[rows]).astype(np.float64)


# ----------------------------------------------------------------------------
# M-matrix filter (Eq. 8 with Eq. 4; Alg. 1, first two steps)
# ----------------------------------------------------------------------------


def row_sums_in_order(A):
    """Row sums of a CSR matrix accumulated left to right in column order
    (Eq. 4 fixes no order; this one is the reading both sides use)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    lens = np.diff(A.indptr)
    if A.nnz == 0:
        return np.zeros(n)
    pos = np.arange(A.nnz) - np.repeat(A.indptr[:-1], lens)
    M = np.zeros((n, int(lens.max())))
    M[np.repeat(np.arange(n), lens), pos] = A.data
    return np.cumsum(M, axis=1)[:, -1]  # trailing zeros leave the sum unchanged


def mmatrix_filter(A):
    """Filtered operator of Alg. 1: A_hat = min(A, 0) entrywise, then
    A_hat <- A_hat - diag(rowsum(A_hat)), so every row sums to zero and the
    off-diagonals are non-positive (Eq. 8 then Eq. 4). Same pattern as A."""
    A = sp.csr_matrix(A, copy=True)
    A.sort_indices()
    Ah = A.copy()
    Ah.data = np.minimum(A.data, 0.0)
    rowsum = row_sums_in_order(Ah)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    on_diag = A.indices == rows
    Ah.data[on_diag] -= rowsum[rows[on_diag]]
    return Ah


def sdc_blocks(indptr, indices, blocks):
    """Separate-displacement-component approximation (Eq. 19-20, Remark 2):
    from a 3x3-block CSR matrix keep, for each component l, the scalar matrix
    A_ll made of the (l, l) entry of every block."""
    n = len(indptr) - 1
    return [sp.csr_matrix((blocks[:, l, l].copy(), indices.copy(), indptr.copy()), shape=(n, n))
            for l in range(3)]


def bsr_to_csr(indptr, indices, blocks):
    """Scalar CSR of a 3x3-block CSR matrix, dof = 3*node + component."""
    n = len(indptr) - 1
    B = sp.bsr_matrix((blocks, indices, indptr), shape=(3 * n, 3 * n)).tocsr()
    B.sort_indices()
    return B


# ----------------------------------------------------------------------------
# restricted smoothing of the basis (Eq. 5-6, Alg. 1)
# ----------------------------------------------------------------------------


def _on_pattern(Q, pat):
    """Values of sparse Q at the entries of the pattern (zeros where absent)."""
    rows = np.repeat(np.arange(pat.shape[0]), np.diff(pat.indptr))
    return np.asarray(Q.tocsr()[rows, pat.indices]).ravel()


def enhanced_msrsb(Ahat, pat, P0, skel, omega=2.0 / 3.0, tol=1e-3, n_it=10, max_iter=100):
    """Alg. 1 (EnhancedMsRSB) on an already filtered operator.

    Each pass: dP = -omega * D_hat^-1 * A_hat * P (Eq. 6); entries of dP outside
    P's fixed support pattern are dropped, so the basis cannot grow beyond its
    support region (the rescaling below restores partition of unity instead of
    moving the overflow to neighbouring bases); P <- P + dP; every row of P is
    divided by its sum; when k mod n_it == 0, e_it is the largest |dP_ij| over
    rows i that are not on the skeleton (support edges). The loop runs while
    e_it > tol and at most max_iter passes. Rows with D_hat_ii = 0 (no
    off-diagonal left after filtering) get dP = 0.
    Returns (vals, iterations, e_it, history of (k, e_it)).
    """
    Ahat = sp.csr_matrix(Ahat)
    n, nc = pat.shape
    dhat = Ahat.diagonal()
    inv = np.zeros(n)
    nz = dhat != 0.0
    inv[nz] = 1.0 / dhat[nz]
    rows = np.repeat(np.arange(n), np.diff(pat.indptr))
    interior = ~skel[rows]
    vals = P0.astype(np.float64).copy()
    k = 0
    e_it = np.inf
    hist = []
    while e_it > tol and k < max_iter:
        vals, dPv = smoothing_pass(Ahat, pat, vals, inv, omega, rows)
        if k % n_it == 0:
            e_it = float(np.max(np.abs(dPv[interior]))) if interior.any() else 0.0
            hist.append((k, e_it))
        k += 1
    return vals, k, e_it, hist


def smoothing_pass(Ahat, pat, vals, inv, omega, rows=None):
    """One pass of Alg. 1's loop body: dP = -omega D_hat^-1 A_hat P (Eq. 6)
    kept on P's pattern, P + dP, rows divided by their sums. inv = 1/D_hat_ii
    (0 where D_hat_ii = 0). Returns (new values, dP on the pattern)."""
    n, nc = pat.shape
    if rows is None:
        rows = np.repeat(np.arange(n), np.diff(pat.indptr))
    P = sp.csr_matrix((vals, pat.indices, pat.indptr), shape=(n, nc))
    AP = Ahat @ P
    dP = -omega * (sp.diags(inv) @ AP)
    dPv = _on_pattern(dP, pat)
    new = vals + dPv
    rs = np.bincount(rows, weights=new, minlength=n)
    return new / rs[rows], dPv


def inverse_diagonal(Ahat):
    d = sp.csr_matrix(Ahat).diagonal()
    inv = np.zeros_like(d)
    inv[d != 0.0] = 1.0 / d[d != 0.0]
    return inv


def as_matrix(vals, pat):
    return sp.csr_matrix((vals, pat.indices, pat.indptr), shape=pat.shape)


def block_prolongation(Ps):
    """Block-diagonal P of the SDC extension (Sec. 4): component l of fine node
    i is interpolated from component l of the coarse nodes only. Rows are
    3*node + l, columns 3*J + l."""
    n, nc = Ps[0].shape
    blocks = []
    for l, P in enumerate(Ps):
        P = sp.coo_matrix(P)
        blocks.append(sp.coo_matrix((P.data, (3 * P.row + l, 3 * P.col + l)), shape=(3 * n, 3 * nc)))
    return sp.csr_matrix(blocks[0] + blocks[1] + blocks[2])


# ----------------------------------------------------------------------------
# Galerkin coarse operator and coarse solver (Eq. 2-3, Alg. 2)
# ----------------------------------------------------------------------------


def galerkin(A, P):
    """A_c = R A P with R = P^T (Galerkin restriction, Sec. 2), unfiltered A."""
    P = sp.csr_matrix(P)
    return (P.T @ (sp.csr_matrix(A) @ P)).tocsr()


def coarse_factor(Ac):
    """M_c^-1 = A_c^-1 through an LU factorisation with partial pivoting (Alg. 2)."""
    return sla.lu_factor(Ac.toarray() if sp.issparse(Ac) else Ac)


def coarse_solve(lu, vc):
    return sla.lu_solve(lu, vc)


# ----------------------------------------------------------------------------
# smoothers (second stage): multicolour orderings, ILU(0), Gauss-Seidel
# ----------------------------------------------------------------------------


def parity_colours(dims):
    """Colour of every grid point: sum_a (x_a mod 2) 2^a. Points of one colour
    never share a 3^d stencil, so each colour class is an independent set."""
    d = len(dims)
    coords = np.indices(dims).reshape(d, -1, order="F")
    col = np.zeros(coords.shape[1], dtype=np.int64)
    for a in range(d):
        col += (coords[a] % 2) << a
    return col


def colour_order(colour):
    """Elimination order: by colour, then by natural index (stable sort)."""
    return np.argsort(colour, kind="stable")


def line_block_order(dims):
    """Elimination order by line blocks: the grid is cut into blocks of whole
    x-lines, 2 lines high in y (and 2 deep in z in 3D); blocks are coloured by
    the parity of their y (and z) block index (2 colours in 2D, 4 in 3D), so
    blocks of one colour never share a 3^d stencil; the order is colour, then
    block, then the natural order inside the block (x fastest). Returns
    (order, colour of every point, block of every point, sub-line of every
    point inside its block)."""
    d = len(dims)
    coords = np.indices(dims).reshape(d, -1, order="F")
    nbk = [-(-dims[a] // 2) for a in range(1, d)]
    colour = np.zeros(coords.shape[1], dtype=np.int64)
    block = np.zeros(coords.shape[1], dtype=np.int64)
    sub = np.zeros(coords.shape[1], dtype=np.int64)
    st = 1
    for a in range(1, d):
        colour += ((coords[a] // 2) % 2) << (a - 1)
        block += (coords[a] // 2) * st
        sub += (coords[a] % 2) << (a - 1)
        st *= nbk[a - 1]
    order = np.lexsort((coords[0], sub, block, colour))
    return order, colour, block, sub


_lib = None


def _native():
    global _lib
    if _lib is None:
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "ilu0.c")
        so = os.path.join(here, "libilu0_oracle.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", so, src])
        _lib = ctypes.CDLL(so)
        _lib.oracle_ilu0.restype = ctypes.c_long
    return _lib


def ilu0(B):
    """ILU(0) of B in B's own row order (pass B already permuted into the
    elimination order). Returns (L unit-lower CSR without its diagonal, U CSR
    with diagonal), both in B's pattern. Raises on a zero pivot."""
    B = sp.csr_matrix(B, copy=True)
    B.sort_indices()
    n = B.shape[0]
    ip = B.indptr.astype(np.int64)
    ix = B.indices.astype(np.int64)
    a = np.ascontiguousarray(B.data, dtype=np.float64)
    lu = np.empty_like(a)
    dpos = np.empty(n, dtype=np.int64)
    work = np.empty(n, dtype=np.int64)
    P = ctypes.POINTER
    r = _native().oracle_ilu0(ctypes.c_int64(n), ip.ctypes.data_as(P(ctypes.c_int64)),
                              ix.ctypes.data_as(P(ctypes.c_int64)), a.ctypes.data_as(P(ctypes.c_double)),
                              lu.ctypes.data_as(P(ctypes.c_double)), dpos.ctypes.data_as(P(ctypes.c_int64)),
                              work.ctypes.data_as(P(ctypes.c_int64)))
    if r != 0:
        raise ZeroDivisionError("ILU(0) zero pivot at row %d" % (r - 1))
    F = sp.csr_matrix((lu, B.indices.copy(), B.indptr.copy()), shape=B.shape)
    L = sp.tril(F, k=-1, format="csr")
    U = sp.triu(F, k=0, format="csr")
    return L, U


class ColouredSmoother:
    """Second-stage smoother (ILU(0), Sec. 3.2; block Gauss-Seidel, Sec. 4.2-4.3).

    kind 'ilu0': M = L U, the ILU(0) factors of A in the elimination order;
    for a symmetric positive definite A these are the IC(0) factors
    (U = diag(U) L^T), the incomplete Cholesky smoother of Sec. 4.1 and 4.3.
    With bdim > 1 the order keeps the dofs of a node together (nodes by
    colour, components inside a node).
    kind 'gs_fwd' / 'gs_bwd': block Gauss-Seidel, M = D + L (forward) or
    M = D + U (backward) of A in the elimination order, with D the
    bdim x bdim diagonal blocks.

    The paper's MATLAB setting eliminates in the natural order (colour=None
    here): the triangular solves are sequential substitutions. With a colour
    array, the order is colour by colour, natural inside a colour (the order
    the GPU uses); the rows of one colour are independent, so each colour is
    one vectorised update, which is exactly sequential substitution in that
    order.
    """

    def __init__(self, A, colour, kind, bdim=1, order=None):
        """colour: per-point colours (colour order), or None with order None
        (natural order); order: an explicit elimination order of the points
        (e.g. line_block_order), solved by sequential substitution."""
        self.kind = kind
        self.bdim = bdim
        A = sp.csr_matrix(A)
        # sequential substitution unless the order is by independent colours
        self.natural = colour is None or order is not None
        if colour is None:
            colour = np.zeros(A.shape[0] // bdim, dtype=np.int64)
        node_order = colour_order(colour) if order is None else np.asarray(order)
        if bdim == 1:
            order = node_order
            dof_colour = colour
        else:
            order = (bdim * node_order[:, None] + np.arange(bdim)[None, :]).ravel()
            dof_colour = np.repeat(colour, bdim)
        self.order = order
        self.inv_order = np.argsort(order)
        B = A[order][:, order].tocsr()
        B.sort_indices()
        self.B = B
        cs = dof_colour[order]
        self.ncol = int(cs.max()) + 1
        self.cls = [np.flatnonzero(cs == c) for c in range(self.ncol)]
        if kind == "ilu0":
            self.L, self.U = ilu0(B)
            self.udiag = self.U.diagonal()
            self.Ustrict = sp.triu(self.U, k=1, format="csr")
        else:
            nn = B.shape[0] // bdim
            node_of = np.arange(B.shape[0]) // bdim
            Bc = B.tocoo()
            same = node_of[Bc.row] == node_of[Bc.col]
            lo = ~same & (Bc.row > Bc.col)
            up = ~same & (Bc.row < Bc.col)
            self.Lo = sp.csr_matrix((Bc.data[lo], (Bc.row[lo], Bc.col[lo])), shape=B.shape)
            self.Up = sp.csr_matrix((Bc.data[up], (Bc.row[up], Bc.col[up])), shape=B.shape)
            blocks = np.zeros((nn, bdim, bdim))
            blocks[node_of[Bc.row[same]], Bc.row[same] % bdim, Bc.col[same] % bdim] = Bc.data[same]
            self.Dinv = np.linalg.inv(blocks)
            self.node_cls = [np.unique(node_of[c]) for c in self.cls]
            if self.natural:
                # (D + T) z = r  <=>  (I + T D^-1) (D z) = r, and T D^-1 keeps
                # T's strict block triangle, so one unit triangular solve
                # followed by the block-diagonal product gives z
                Dm = sp.bsr_matrix((self.Dinv, np.arange(nn), np.arange(nn + 1)), shape=B.shape).tocsr()
                T = self.Lo if kind == "gs_fwd" else self.Up
                self.Dm = Dm
                self.TD = sp.csr_matrix(T @ Dm)
                self.TD.sort_indices()

    def solve(self, r):
        """z = M^-1 r (r, z in the natural order)."""
        rp = r[self.order]
        if self.natural or (self.kind == "ilu0" and self.bdim > 1):
            # sequential substitution (dofs of one node are coupled, so a
            # colour class is not an independent set when bdim > 1)
            if self.kind == "ilu0":
                y = spla.spsolve_triangular(self.L, rp, lower=True, unit_diagonal=True)
                z = spla.spsolve_triangular(self.U, y, lower=False)
            else:
                y = spla.spsolve_triangular(self.TD, rp, lower=self.kind == "gs_fwd", unit_diagonal=True)
                z = self.Dm @ y
            return z[self.inv_order]
        if self.kind == "ilu0":
            y = np.zeros_like(rp)
            for c in range(self.ncol):  # L y = r, unit lower
                idx = self.cls[c]
                y[idx] = rp[idx] - self.L[idx] @ y
            z = np.zeros_like(rp)
            for c in reversed(range(self.ncol)):  # U z = y
                idx = self.cls[c]
                z[idx] = (y[idx] - self.Ustrict[idx] @ z) / self.udiag[idx]
        else:
            bd = self.bdim
            z = np.zeros_like(rp)
            seq = range(self.ncol) if self.kind == "gs_fwd" else reversed(range(self.ncol))
            T = self.Lo if self.kind == "gs_fwd" else self.Up
            for c in seq:
                idx = self.cls[c]
                rhs = rp[idx] - T[idx] @ z
                nodes = self.node_cls[c]
                z[idx] = np.einsum("nij,nj->ni", self.Dinv[nodes], rhs.reshape(-1, bd)).ravel()
        return z[self.inv_order]


class L1Jacobi:
    """l1-Jacobi smoother, the first of the three pre/post-smoother choices of
    the mechanics experiments (Sec. 4, "2 sweeps of l1-Jacobi"). Reading: the
    pointwise l1 diagonal d_i = sum_j |a_ij| over the scalar row i (for 3x3
    blocks, the row of the expanded scalar matrix); one sweep is
    z <- z + D_l1^-1 (r - A z) from z = 0, and solve(r) returns z after
    `sweeps` sweeps, so M^-1 is a fixed symmetric polynomial in D^-1 A."""

    def __init__(self, A, sweeps=2):
        self.A = sp.csr_matrix(A)
        self.d = np.asarray(abs(self.A).sum(axis=1)).ravel()
        self.sweeps = sweeps

    def solve(self, r):
        z = np.zeros_like(r)
        for _ in range(self.sweeps):
            z = z + (r - self.A @ z) / self.d
        return z


# ----------------------------------------------------------------------------
# two-stage preconditioner (Alg. 3 and Alg. 4)
# ----------------------------------------------------------------------------


def fv_restriction(part, nc, bdim=1):
    """Petrov-Galerkin restriction of Sec. 2 in its finite-volume form (the
    MSFV choice): R_Ji = 1 when fine point i lies in primal coarse block J,
    so the coarse equations are sums of fine equations over each block and
    the coarse problem keeps discrete mass conservation. For bdim > 1 the
    same indicator acts on every component (row bdim*J + l, column
    bdim*i + l). Returns an (nc*bdim) x (n*bdim) CSR matrix."""
    part = np.asarray(part)
    n = len(part)
    rows = (bdim * part[:, None] + np.arange(bdim)[None, :]).ravel()
    cols = (bdim * np.arange(n)[:, None] + np.arange(bdim)[None, :]).ravel()
    return sp.csr_matrix((np.ones(n * bdim), (rows, cols)), shape=(nc * bdim, n * bdim))


class TwoLevel:
    """Alg. 2 set-up pieces bundled for Alg. 3/4: P, the restriction R (P^T,
    the Galerkin choice, unless R is given: e.g. fv_restriction, the
    Petrov-Galerkin choice of Alg. 2), A_c = R A P, M_c^-1 and the optional
    pre/post smoothers (objects with .solve)."""

    def __init__(self, A, P, pre=None, post=None, coarse=True, R=None):
        self.A = sp.csr_matrix(A)
        self.P = sp.csr_matrix(P)
        self.R = self.P.T.tocsr() if R is None else sp.csr_matrix(R)
        self.Ac = (self.R @ (self.A @ self.P)).tocsr() if R is not None else galerkin(self.A, self.P)
        self.lu = coarse_factor(self.Ac)
        self.pre = pre
        self.post = post
        self.coarse = coarse  # False: the smoothing-only baseline of Sec. 3.2 and Sec. 4

    def multiscale(self, v):
        """Alg. 3: v_c = R v; w_c = M_c^-1 v_c; w = P w_c."""
        vc = self.R @ v
        wc = coarse_solve(self.lu, vc)
        return self.P @ wc

    def apply(self, v):
        """Alg. 4 from z = 0: optional pre-smoothing, coarse correction with the
        residual v - A z, optional post-smoothing."""
        z = np.zeros_like(v)
        if self.pre is not None:
            z = z + self.pre.solve(v - self.A @ z)
        if self.coarse:
            z = z + self.multiscale(v - self.A @ z)
        if self.post is not None:
            z = z + self.post.solve(v - self.A @ z)
        return z


# ----------------------------------------------------------------------------
# Krylov accelerators (GMRES, right preconditioned; PCG)
# ----------------------------------------------------------------------------


def gmres_right(A, b, M, x0=None, rtol=1e-8, maxit=200, restart=200):
    """Right-preconditioned GMRES with modified Gram-Schmidt Arnoldi and Givens
    rotations (Saad, Iterative Methods, Alg. 9.5). Stops when the rotated
    residual estimate is <= rtol ||b||; the true residual is then checked and
    the method restarts from the current x if it is not yet met.
    Returns (x, iterations, relres, history of estimated relative residuals)."""
    A = sp.csr_matrix(A)
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0, []
    its = 0
    hist = []
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm or its >= maxit:
            return x, its, beta / bnorm, hist
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        Hh = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = A @ Z[j]
            for i in range(j + 1):
                Hh[i, j] = np.dot(w, V[i])
                w = w - Hh[i, j] * V[i]
            Hh[j + 1, j] = np.linalg.norm(w)
            if Hh[j + 1, j] != 0.0:
                V[j + 1] = w / Hh[j + 1, j]
            for i in range(j):
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -sn[i] * Hh[i, j] + cs[i] * Hh[i + 1, j]
                Hh[i, j] = t
            den = np.hypot(Hh[j, j], Hh[j + 1, j])
            cs[j] = Hh[j, j] / den
            sn[j] = Hh[j + 1, j] / den
            Hh[j, j] = den
            Hh[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm:
                break
        y = sla.solve_triangular(Hh[:j_done, :j_done], g[:j_done])
        x = x + Z[:j_done].T @ y


def richardson(A, b, M, x0=None, rtol=1e-8, maxit=200):
    """Preconditioned Richardson iteration, the stand-alone use of the
    two-stage operator in Sec. 3.2: x <- x + M^-1 (b - A x), stopping when the
    true relative residual is <= rtol. Returns (x, iterations, relres,
    history)."""
    A = sp.csr_matrix(A)
    x = np.zeros(len(b)) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    hist = []
    its = 0
    while True:
        r = b - A @ x
        rr = np.linalg.norm(r) / bnorm
        if its > 0:
            hist.append(rr)
        if rr <= rtol or its >= maxit:
            return x, its, rr, hist
        x = x + M(r)
        its += 1


def pcg(A, b, M, x0=None, rtol=1e-8, maxit=500):
    """Preconditioned conjugate gradients (Saad, Alg. 9.1) with a symmetric
    preconditioner M; stops on the recursively updated residual <= rtol ||b||
    and confirms with the true residual.
    Returns (x, iterations, relres, history)."""
    A = sp.csr_matrix(A)
    x = np.zeros(len(b)) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r = b - A @ x
    hist = []
    its = 0
    if np.linalg.norm(r) <= rtol * bnorm:
        return x, 0, np.linalg.norm(r) / bnorm, hist
    z = M(r)
    p = z.copy()
    rz = np.dot(r, z)
    while its < maxit:
        q = A @ p
        alpha = rz / np.dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        its += 1
        rn = np.linalg.norm(r)
        hist.append(rn / bnorm)
        if rn <= rtol * bnorm:
            rt = np.linalg.norm(b - A @ x)
            if rt <= rtol * bnorm:
                return x, its, rt / bnorm, hist
            r = b - A @ x
        z = M(r)
        rz_new = np.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, its, np.linalg.norm(b - A @ x) / bnorm, hist


# ----------------------------------------------------------------------------
# Whole pipelines (Alg. 2 set-up + Krylov solve), as the library exposes them
# ----------------------------------------------------------------------------


def setup_scalar(A, dims, H, centering=0, omega=2.0 / 3.0, tol=1e-3, n_it=10, max_iter=100,
                 smoother="ilu0", coarse=True, order="lines", restriction="galerkin"):
    """Alg. 2 for a scalar operator (flow): partition, filter, Alg. 1, Galerkin
    coarse operator, coarse LU and an ILU(0) post-smoother, eliminated in the
    parity-colour order (order="colour"), by line blocks (order="lines",
    line_block_order) or in the natural order (order="natural", the paper's
    MATLAB setting). restriction "galerkin"
    (R = P^T) or "fv" (the finite-volume Petrov-Galerkin R of fv_restriction)."""
    A = sp.csr_matrix(A)
    A.sort_indices()
    part = partition(dims, H, centering)
    Ahat = mmatrix_filter(A)
    P0 = indicator(part["part"], part["pat"])
    vals, its, e_it, hist = enhanced_msrsb(Ahat, part["pat"], P0, part["skel"], omega, tol, n_it, max_iter)
    P = as_matrix(vals, part["pat"])
    if order == "lines":
        lo, lcol, _, _ = line_block_order(dims)
        post = ColouredSmoother(A, lcol, "ilu0", order=lo) if smoother == "ilu0" else None
    else:
        col = parity_colours(dims) if order == "colour" else None
        post = ColouredSmoother(A, col, "ilu0") if smoother == "ilu0" else None
    R = fv_restriction(part["part"], part["nc"]) if restriction == "fv" else None
    tl = TwoLevel(A, P, pre=None, post=post, coarse=coarse, R=R)
    return dict(part=part, Ahat=Ahat, vals=vals, iters=its, e_it=e_it, hist=hist, P=P, tl=tl)


def setup_elastic(indptr, indices, blocks, dims, H, omega=2.0 / 3.0, tol=1e-3, n_it=10, max_iter=100,
                  smoother="gs", sweeps=2, coarse=True, order="colour"):
    """Alg. 2 for 3x3-block elasticity: SDC blocks filtered per component,
    three scalar bases on one shared pattern, block-diagonal P, Galerkin with
    the full operator, and a symmetric pair of pre/post smoothers: forward /
    backward block Gauss-Seidel ("gs"), or `sweeps` l1-Jacobi sweeps each
    ("l1jac"), or IC(0) ("ic0", Sec. 4.1 and 4.3: M = L L^T-type incomplete
    Cholesky, the same M before and after the coarse stage). coarse=False
    gives the smoothing-only baseline. order as in setup_scalar (Gauss-Seidel
    and IC(0))."""
    part = partition(dims, H, 1)
    A = bsr_to_csr(indptr, indices, blocks)
    comps = sdc_blocks(indptr, indices, blocks)
    P0 = indicator(part["part"], part["pat"])
    out = []
    for l in range(3):
        Ahat = mmatrix_filter(comps[l])
        out.append(enhanced_msrsb(Ahat, part["pat"], P0, part["skel"], omega, tol, n_it, max_iter))
    Ps = [as_matrix(o[0], part["pat"]) for o in out]
    P = block_prolongation(Ps)
    if smoother == "l1jac":
        pre = post = L1Jacobi(A, sweeps)
    elif smoother == "ic0":
        pre = post = ColouredSmoother(A, parity_colours(dims) if order == "colour" else None, "ilu0", bdim=3)
    else:
        col = parity_colours(dims) if order == "colour" else None
        pre = ColouredSmoother(A, col, "gs_fwd", bdim=3)
        post = ColouredSmoother(A, col, "gs_bwd", bdim=3)
    tl = TwoLevel(A, P, pre=pre, post=post, coarse=coarse)
    return dict(part=part, comps=out, P=P, tl=tl, A=A)


# ----------------------------------------------------------------------------
# adjoint gradient of a pressure objective with respect to log-permeability
# ----------------------------------------------------------------------------


def tpfa_objective_gradient(dims, logk, obs, p_obs):
    """J(theta) = sum_o (p[obs_o] - p_obs_o)^2 for the two-point flux system of
    isotropic cells k = exp(theta) (unit cells, face transmissibility
    T = 2 k_L k_R / (k_L + k_R), p = 1 on the x = 0 face and p = 0 on the
    x = nx face through half-cell transmissibility 2 k, no flow elsewhere;
    cells x fastest), and dJ/dtheta by the adjoint method: A p = b,
    A^T lambda = dJ/dp, dJ/dtheta = lambda^T (db/dtheta - dA/dtheta p), with
    dT/dtheta_L = 2 k_L k_R^2 / (k_L + k_R)^2 (and symmetrically for R).
    Direct sparse solves in FP64. Returns (J, grad, p)."""
    dims = tuple(dims)
    d = len(dims)
    n = int(np.prod(dims))
    k = np.exp(np.asarray(logk, dtype=np.float64))
    idx = np.arange(n).reshape(dims[::-1])
    fl, fr = [], []
    for a in range(d):
        ax = d - 1 - a
        fl.append(np.take(idx, np.arange(dims[a] - 1), axis=ax).ravel())
        fr.append(np.take(idx, np.arange(1, dims[a]), axis=ax).ravel())
    fl, fr = np.concatenate(fl), np.concatenate(fr)
    kl, kr = k[fl], k[fr]
    T = 2.0 * kl * kr / (kl + kr)
    west = np.take(idx, [0], axis=d - 1).ravel()
    east = np.take(idx, [dims[0] - 1], axis=d - 1).ravel()
    rows = np.concatenate([fl, fr, fl, fr, west, east])
    cols = np.concatenate([fl, fr, fr, fl, west, east])
    data = np.concatenate([T, T, -T, -T, 2.0 * k[west], 2.0 * k[east]])
    A = sp.csr_matrix((data, (rows, cols)), shape=(n, n))
    b = np.zeros(n)
    np.add.at(b, west, 2.0 * k[west])
    p = spla.spsolve(A.tocsc(), b)
    r = p[obs] - p_obs
    J = float(r @ r)
    gp = np.zeros(n)
    np.add.at(gp, obs, 2.0 * r)
    lam = spla.spsolve(A.T.tocsc(), gp)
    dT_l = 2.0 * kl * kr * kr / (kl + kr) ** 2
    dT_r = 2.0 * kr * kl * kl / (kl + kr) ** 2
    flux = (lam[fl] - lam[fr]) * (p[fl] - p[fr])
    grad = np.zeros(n)
    np.add.at(grad, fl, -dT_l * flux)
    np.add.at(grad, fr, -dT_r * flux)
    np.add.at(grad, west, 2.0 * k[west] * lam[west] * (1.0 - p[west]))
    np.add.at(grad, east, -2.0 * k[east] * lam[east] * p[east])
    return J, grad, p


# ----------------------------------------------------------------------------
# adjoint gradient through MPFA-O (3D, unit cells): dJ/d ln k per cell
# ----------------------------------------------------------------------------


def mpfa_region_parts(K, dims):
    """The interaction regions of MPFA-O (continuity points at the half-face
    midpoints) on a 3D grid of unit cells with no-flow outer faces, split by
    cell: for every grid vertex (C order over the (nx+1, ny+1, nz+1) vertex
    grid) and each of its 8 cell slots s (offset o in {0,1}^3, cell = vertex -
    1 + o), the K-dependent parts C_s, D_s, G_s, H_s of the local system
    C u = D p, half-face fluxes F = G u + H p (C also has a constant identity
    part on half-faces with no cell). Half-face f (axis a, minus slot, plus
    slot) carries the flux from its minus cell to its plus cell. Per cell s,
    the linear reconstruction through the cell pressure and the potentials u
    at the midpoints of its 3 half-faces gives the flux across its half-face
    normal to axis a: sum_b U[a, b] (u_b - p_s), U = -2 (1/4) K_s sign_b.
    Returns dict(C0, Cs, Ds, Gs, Hs, cells, present, faces)."""
    d = 3
    nv = tuple(s + 1 for s in dims)
    nvert = int(np.prod(nv))
    offs = [(i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    loc = {o: s for s, o in enumerate(offs)}
    faces = []
    for a in range(d):
        for q0 in (0, 1):
            for q1 in (0, 1):
                q = [q0, q1]
                om = tuple(q[:a] + [0] + q[a:])
                op = tuple(q[:a] + [1] + q[a:])
                faces.append((a, loc[om], loc[op]))
    fof = {}  # (slot, axis) -> half-face
    for f, (a, sm, sp_) in enumerate(faces):
        fof[(sm, a)] = f
        fof[(sp_, a)] = f
    V = np.indices(nv).reshape(d, -1)
    cells = np.zeros((nvert, 8), dtype=np.int64)
    present = np.zeros((nvert, 8), dtype=bool)
    Kc = np.zeros((nvert, 8, 3, 3))
    for s, o in enumerate(offs):
        cc = [V[a] - 1 + o[a] for a in range(d)]
        ok = np.ones(nvert, dtype=bool)
        for a in range(d):
            ok &= (cc[a] >= 0) & (cc[a] < dims[a])
        present[:, s] = ok
        ci = [np.clip(cc[a], 0, dims[a] - 1) for a in range(d)]
        cells[:, s] = ci[0] + dims[0] * (ci[1] + dims[1] * ci[2])
        Kc[:, s] = K[ci[0], ci[1], ci[2]] * ok[:, None, None]
    sign = np.array([[1.0 if o[b] == 0 else -1.0 for b in range(d)] for o in offs])
    U = -2.0 * 0.25 * Kc * sign[None, :, None, :]  # (nvert, slot, a, b)
    nf = 12
    C0 = np.zeros((nvert, nf, nf))
    Cs = np.zeros((8, nvert, nf, nf))
    Ds = np.zeros((8, nvert, nf, 8))
    Gs = np.zeros((8, nvert, nf, nf))
    Hs = np.zeros((8, nvert, nf, 8))
    for f, (a, sm, sp_) in enumerate(faces):
        pm, pp = present[:, sm], present[:, sp_]
        both = pm & pp
        only_m, only_p = pm & ~pp, pp & ~pm
        # continuity F_m = F_p, or no flow F = 0 from the one present cell
        use_m = both | only_m
        for b in range(d):
            Cs[sm, :, f, fof[(sm, b)]] += use_m * U[:, sm, a, b]
            Cs[sp_, :, f, fof[(sp_, b)]] -= both * U[:, sp_, a, b]
            Cs[sp_, :, f, fof[(sp_, b)]] += only_p * U[:, sp_, a, b]
        Ds[sm, :, f, sm] += use_m * U[:, sm, a, :].sum(axis=1)
        Ds[sp_, :, f, sp_] -= both * U[:, sp_, a, :].sum(axis=1)
        Ds[sp_, :, f, sp_] += only_p * U[:, sp_, a, :].sum(axis=1)
        C0[:, f, f] += ~(pm | pp)
        # the half-face flux, from the minus cell if present
        gm, gp = pm, ~pm & pp
        for b in range(d):
            Gs[sm, :, f, fof[(sm, b)]] += gm * U[:, sm, a, b]
            Gs[sp_, :, f, fof[(sp_, b)]] += gp * U[:, sp_, a, b]
        Hs[sm, :, f, sm] -= gm * U[:, sm, a, :].sum(axis=1)
        Hs[sp_, :, f, sp_] -= gp * U[:, sp_, a, :].sum(axis=1)
    return dict(C0=C0, Cs=Cs, Ds=Ds, Gs=Gs, Hs=Hs, cells=cells, present=present, faces=faces)


def mpfa_lam_dA_p(parts, lam, p):
    """g_c = lam^T (dA/d ln k_c) p for the MPFA-O matrix of a grid of unit
    cells with no-flow outer faces (K_c = k_c K_hat_c, so dK_c/d ln k_c = K_c
    and each local matrix's cell-c part is its derivative). Per interaction
    region: u = C^-1 D p, w_f = lam(minus cell) - lam(plus cell) on half-faces
    between two cells (no-flow half-faces carry no flux), mu = C^-T G^T w, and
    the region adds w^T (G_c u + H_c p) + mu^T (D_c p - C_c u) to cell c."""
    C = parts["C0"] + parts["Cs"].sum(axis=0)
    D = parts["Ds"].sum(axis=0)
    G = parts["Gs"].sum(axis=0)
    cells, present = parts["cells"], parts["present"]
    pl = np.where(present, p[cells], 0.0)
    ll = np.where(present, lam[cells], 0.0)
    w = np.zeros((cells.shape[0], 12))
    for f, (a, sm, sp_) in enumerate(parts["faces"]):
        both = present[:, sm] & present[:, sp_]
        w[:, f] = both * (ll[:, sm] - ll[:, sp_])
    u = np.linalg.solve(C, np.einsum("vfc,vc->vf", D, pl)[..., None])[..., 0]
    Gtw = np.einsum("vgf,vg->vf", G, w)
    mu = np.linalg.solve(np.transpose(C, (0, 2, 1)), Gtw[..., None])[..., 0]
    g = np.zeros(len(p))
    for s in range(8):
        t = (np.einsum("vf,vfg,vg->v", w, parts["Gs"][s], u) + np.einsum("vf,vfc,vc->v", w, parts["Hs"][s], pl)
             + np.einsum("vf,vfc,vc->v", mu, parts["Ds"][s], pl) - np.einsum("vf,vfg,vg->v", mu, parts["Cs"][s], u))
        np.add.at(g, cells[present[:, s], s], t[present[:, s]])
    return g


def mpfa_objective_gradient(K_hat, logk, wells, obs, p_obs, A=None, b=None):
    """J(theta) = sum_o (p[obs_o] - p_obs_o)^2 for MPFA-O Darcy flow on unit
    cells with K_c = exp(theta_c) K_hat_c, no-flow outer faces and
    bottom-hole-pressure wells (A_ii += WI_i, b_i = WI_i p_w, WI_i = the MPFA-O
    diagonal A_ii), and dJ/dtheta by the adjoint method: A p = b,
    A^T lambda = dJ/dp = 2 (p - p_obs) on the observation cells, and
    dJ/dtheta_c = -lambda^T (dA/dtheta_c) p + lambda^T db/dtheta_c, where the
    wells add -lambda_i (p_i - p_w) dA_ii/dtheta_c. A, b (optional) are the
    assembled system at theta (scipy CSR, vector). Direct sparse solves in
    FP64. Returns (J, grad, p)."""
    dims = K_hat.shape[:3]
    K = np.exp(np.asarray(logk)).reshape(dims, order="F")[..., None, None] * K_hat
    parts = mpfa_region_parts(K, dims)
    if A is None:
        raise ValueError("pass the assembled system (A, b)")
    A = sp.csr_matrix(A)
    p = spla.spsolve(A.tocsc(), b)
    r = p[obs] - p_obs
    J = float(r @ r)
    gp = np.zeros(len(p))
    np.add.at(gp, obs, 2.0 * r)
    lam = spla.spsolve(A.T.tocsc(), gp)
    grad = -mpfa_lam_dA_p(parts, lam, p)
    n = len(p)
    for cell, pw in wells:
        e = np.zeros(n)
        e[cell] = 1.0
        grad -= lam[cell] * (p[cell] - pw) * mpfa_lam_dA_p(parts, e, e)
    return J, grad, p
