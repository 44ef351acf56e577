"""Finite-volume Darcy operators on uniform Cartesian grids of unit cells.

The fine-scale pressure system A p = b of -div(K grad p) = q is assembled with
the MPFA-O method (the multipoint scheme the paper's flow cases use) or with TPFA
(the two-point scheme, exact for K-orthogonal grids). Cells are ordered with x
fastest: flat = i0 + n0*(i1 + n1*i2). Each cell equation is the sum of fluxes
leaving the cell, so A has a positive diagonal.

Boundary conditions are given per domain side, ``bc[(axis, side)]`` with side 0 =
low (x_axis = 0) and 1 = high, as ``("D", value)`` for a fixed pressure or
``("N",)`` for no flow (the default).
"""
import itertools

import numpy as np
import scipy.sparse as sp

from .fields import gaussian_random_field, rotation_2d, rotation_zyx


def _stencil_offsets(d):
    # offsets in {-1,0,1}^d, x fastest (itertools varies the last entry fastest)
    return [tuple(reversed(t)) for t in itertools.product((-1, 0, 1), repeat=d)]


def _stencil_to_csr(dims, A_st):
    """Convert a per-cell stencil array (*dims, 3^d) to CSR, keeping every
    in-domain neighbour (the structural 3^d pattern) with sorted columns."""
    d = len(dims)
    n = int(np.prod(dims))
    offs = _stencil_offsets(d)
    coords = np.indices(dims).reshape(d, -1, order="F")  # (d, n) in flat order
    flat = np.arange(n)
    strides = [int(np.prod(dims[:a])) for a in range(d)]
    rows, cols, vals = [], [], []
    A_flat = _grid_flat(A_st, dims)
    for s, o in enumerate(offs):
        ok = np.ones(n, dtype=bool)
        shift = 0
        for a in range(d):
            c = coords[a] + o[a]
            ok &= (c >= 0) & (c < dims[a])
            shift += o[a] * strides[a]
        r = flat[ok]
        rows.append(r)
        cols.append(r + shift)
        vals.append(A_flat[ok, s])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


def _grid_flat(a, dims):
    """Flatten a (*dims, ...) array to (n, ...) with x fastest."""
    n = int(np.prod(dims))
    rest = a.shape[len(dims):]
    return np.moveaxis(a, list(range(len(dims))), list(reversed(range(len(dims))))).reshape((n,) + rest)


def mpfa_o(K, bc=None, wells=None):
    """MPFA-O (eta = 0) on a uniform Cartesian grid of unit cells.

    K : array (*dims, d, d), symmetric positive-definite cell tensors.
    In every interaction region (the 2^d cells around a grid vertex) the pressure
    is linear per cell, fixed by the cell pressure and the potentials at the
    midpoints of the cell's d faces touching the vertex; flux continuity on each
    of the d*2^(d-1) half-faces (or the boundary condition there) gives a local
    system whose solution expresses every half-face flux in the cell pressures.
    Returns (indptr, indices, data, b) with int32 CSR and float64 values.
    """
    bc = bc or {}
    K = np.asarray(K, dtype=np.float64)
    dims = K.shape[:-2]
    d = len(dims)
    assert K.shape[-2:] == (d, d)
    nv = tuple(s + 1 for s in dims)
    nvert = int(np.prod(nv))
    offs = list(itertools.product((0, 1), repeat=d))  # local cells of a region
    ncell = len(offs)
    loc = {o: c for c, o in enumerate(offs)}
    area = 0.5 ** (d - 1)

    # half-faces: axis a, offsets q of the other axes
    faces = []
    for a in range(d):
        for q in itertools.product((0, 1), repeat=d - 1):
            om = tuple(list(q[:a]) + [0] + list(q[a:]))
            op = tuple(list(q[:a]) + [1] + list(q[a:]))
            faces.append((a, loc[om], loc[op]))
    nf = len(faces)
    fidx = {}
    for f, (a, cm, cp) in enumerate(faces):
        fidx[(cm, a)] = f
        fidx[(cp, a)] = f

    V = np.indices(nv).reshape(d, -1)  # vertex coords, C order over nv
    pres = np.zeros((nvert, ncell), dtype=bool)
    Kc = np.zeros((nvert, ncell, d, d))
    for c, o in enumerate(offs):
        cc = [V[a] - 1 + o[a] for a in range(d)]
        ok = np.ones(nvert, dtype=bool)
        for a in range(d):
            ok &= (cc[a] >= 0) & (cc[a] < dims[a])
        pres[:, c] = ok
        idx = tuple(np.clip(cc[a], 0, dims[a] - 1) for a in range(d))
        Kc[:, c] = K[idx] * ok[:, None, None]

    # flux F_c(a) across the half-face of cell c normal to axis a (in +a
    # direction) = sum_b U[c,a,b] * u_{f(c,b)} + Pc[c,a] * p_c
    s = np.array([[1.0 if o[a] == 0 else -1.0 for a in range(d)] for o in offs])  # (ncell, d)
    U = -2.0 * area * Kc * s[None, :, None, :]  # (nvert, ncell, a, b)
    Pc = -U.sum(axis=3)  # (nvert, ncell, a)

    C = np.zeros((nvert, nf, nf))
    D = np.zeros((nvert, nf, ncell))
    e = np.zeros((nvert, nf))
    G = np.zeros((nvert, nf, nf))
    Hm = np.zeros((nvert, nf, ncell))
    side_val = {}
    for f, (a, cm, cp) in enumerate(faces):
        pm, pp = pres[:, cm], pres[:, cp]
        both = pm & pp
        only_m = pm & ~pp  # vertex on the high side of axis a
        only_p = pp & ~pm  # vertex on the low side of axis a
        none = ~pm & ~pp
        kind_hi = bc.get((a, 1), ("N",))
        kind_lo = bc.get((a, 0), ("N",))
        dir_m = only_m & (kind_hi[0] == "D")
        dir_p = only_p & (kind_lo[0] == "D")
        neu_m = only_m & (kind_hi[0] != "D")
        neu_p = only_p & (kind_lo[0] != "D")
        ident = none | dir_m | dir_p
        for b in range(d):
            C[:, f, fidx[(cm, b)]] += (both | neu_m) * U[:, cm, a, b]
            C[:, f, fidx[(cp, b)]] -= both * U[:, cp, a, b]
            C[:, f, fidx[(cp, b)]] += neu_p * U[:, cp, a, b]
        D[:, f, cm] -= (both | neu_m) * Pc[:, cm, a]
        D[:, f, cp] += both * Pc[:, cp, a]
        D[:, f, cp] -= neu_p * Pc[:, cp, a]
        C[:, f, f] += ident
        if kind_hi[0] == "D":
            e[:, f] += dir_m * kind_hi[1]
        if kind_lo[0] == "D":
            e[:, f] += dir_p * kind_lo[1]
        # flux from the minus cell if present, else the plus cell
        use_m = pm
        use_p = ~pm & pp
        for b in range(d):
            G[:, f, fidx[(cm, b)]] += use_m * U[:, cm, a, b]
            G[:, f, fidx[(cp, b)]] += use_p * U[:, cp, a, b]
        Hm[:, f, cm] += use_m * Pc[:, cm, a]
        Hm[:, f, cp] += use_p * Pc[:, cp, a]
        side_val[f] = (both, only_m & ~neu_m, only_p & ~neu_p)

    Cinv_D = np.linalg.solve(C, D)
    Cinv_e = np.linalg.solve(C, e[..., None])[..., 0]
    T = np.einsum("vfg,vgc->vfc", G, Cinv_D) + Hm  # (nvert, nf, ncell)
    t = np.einsum("vfg,vg->vf", G, Cinv_e)  # (nvert, nf)

    n3 = 3 ** d
    offs3 = _stencil_offsets(d)
    st_index = {o: k for k, o in enumerate(offs3)}
    A_st = np.zeros(tuple(dims) + (n3,))
    bgrid = np.zeros(tuple(dims))
    Tg = T.reshape(tuple(nv) + (nf, ncell))
    tg = t.reshape(tuple(nv) + (nf,))

    def add(row_off, sign, f, use_mask):
        # rows: cell at v - 1 + row_off, over vertices where that cell exists
        vsl = tuple(slice(1 - row_off[a], nv[a] - row_off[a]) for a in range(d))
        csl = tuple(slice(0, dims[a]) for a in range(d))
        m = use_mask.reshape(nv)[vsl]
        for c, o in enumerate(offs):
            rel = tuple(o[a] - row_off[a] for a in range(d))
            A_st[csl + (st_index[rel],)] += sign * m * Tg[vsl + (f, c)]
        bgrid[csl] -= sign * m * tg[vsl + (f,)]

    for f, (a, cm, cp) in enumerate(faces):
        both, bnd_m, bnd_p = side_val[f]
        add(offs[cm], +1.0, f, both | bnd_m)
        add(offs[cp], -1.0, f, both | bnd_p)

    indptr, indices, data = _stencil_to_csr(dims, A_st)
    b = _grid_flat(bgrid, dims).copy()
    if wells:
        _add_wells(indptr, indices, data, b, wells)
    return indptr, indices, data, b


def _add_wells(indptr, indices, data, b, wells):
    """Bottom-hole-pressure wells: A_ii += WI, b_i += WI * p_w with WI = A_ii."""
    for cell, pw in wells:
        lo, hi = indptr[cell], indptr[cell + 1]
        k = lo + int(np.searchsorted(indices[lo:hi], cell))
        wi = data[k]
        data[k] += wi
        b[cell] += wi * pw


def tpfa(K, bc=None, wells=None):
    """Two-point flux approximation on unit cells (uses the diagonal of K only).

    Face transmissibility is the harmonic mean 2 k1 k2 / (k1 + k2) of the two
    cells' diagonal entries; a fixed-pressure boundary face has 2 k. The pattern
    is the same 3^d structural pattern mpfa_o returns (unused entries are 0).
    """
    bc = bc or {}
    K = np.asarray(K, dtype=np.float64)
    dims = K.shape[:-2]
    d = len(dims)
    offs3 = _stencil_offsets(d)
    st_index = {o: k for k, o in enumerate(offs3)}
    A_st = np.zeros(tuple(dims) + (3 ** d,))
    bgrid = np.zeros(tuple(dims))
    ctr = st_index[(0,) * d]
    for a in range(d):
        ka = K[..., a, a]
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[a] = slice(0, dims[a] - 1)
        hi[a] = slice(1, dims[a])
        k1, k2 = ka[tuple(lo)], ka[tuple(hi)]
        T = 2.0 * k1 * k2 / (k1 + k2)
        plus = tuple(1 if b == a else 0 for b in range(d))
        minus = tuple(-1 if b == a else 0 for b in range(d))
        A_st[tuple(lo) + (ctr,)] += T
        A_st[tuple(lo) + (st_index[plus],)] -= T
        A_st[tuple(hi) + (ctr,)] += T
        A_st[tuple(hi) + (st_index[minus],)] -= T
        for side in (0, 1):
            kind = bc.get((a, side), ("N",))
            if kind[0] != "D":
                continue
            sl = [slice(None)] * d
            sl[a] = slice(0, 1) if side == 0 else slice(dims[a] - 1, dims[a])
            sl = tuple(sl)
            A_st[sl + (ctr,)] += 2.0 * ka[sl]
            bgrid[sl] += 2.0 * ka[sl] * kind[1]
    indptr, indices, data = _stencil_to_csr(dims, A_st)
    b = _grid_flat(bgrid, dims).copy()
    if wells:
        _add_wells(indptr, indices, data, b, wells)
    return indptr, indices, data, b


def anisotropic_tensors(logk, R, ratios):
    """Per-cell K = R diag(k * ratios) R^T with k = exp(logk)."""
    k = np.exp(logk)
    Dg = np.asarray(ratios, dtype=np.float64)
    base = R @ np.diag(Dg) @ R.T
    return k[..., None, None] * base


def pattern27(dims):
    """CSR pattern (int32) of every cell's in-grid 3x3x3 neighbours on a 3D
    grid (cells x fastest), columns ascending: the structural pattern of the
    MPFA-O operators above."""
    nx, ny, nz = dims
    n = nx * ny * nz
    i = np.arange(n)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    cols = np.full((n, 27), -1, dtype=np.int64)
    for q in range(27):
        dx, dy, dz = q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & (z + dz >= 0) & (z + dz < nz)
        cols[ok, q] = i[ok] + dx + nx * (dy + ny * dz)
    rowptr = np.concatenate([[0], np.cumsum((cols >= 0).sum(axis=1))]).astype(np.int32)
    return rowptr, cols[cols >= 0].astype(np.int32)


def darcy_3d_field(dims, seed, sigma=3.0, corr_len=8.0):
    """The inputs of the 3D MPFA-O case without its assembly: ln k (cells x
    fastest; the Gaussian random field of darcy_3d_case from the same seed),
    the unit anisotropy tensors K_hat [n][3][3] (10:1, rotated (20, 35, 0)
    degrees) and the corner well pair, for assembling on the device."""
    rng = np.random.default_rng(seed)
    logk = gaussian_random_field(tuple(dims), corr_len, sigma, rng)
    n = int(np.prod(dims))
    K_hat = anisotropic_tensors(np.zeros(tuple(dims)), rotation_zyx(20.0, 35.0, 0.0), (1.0, 1.0, 0.1))
    K_hat = np.ascontiguousarray(np.moveaxis(K_hat, [0, 1, 2], [2, 1, 0]).reshape(n, 3, 3))
    return logk.ravel(order="F"), K_hat, [(0, 1.0), (n - 1, 0.0)]


def darcy_2d_case(n=64, H=8, seed=1001):
    """2D MPFA-O case: ln k i.i.d. N(0,1), K = R(30) diag(k, 0.1k) R(30)^T,
    p = 1 at x = 0, p = 0 at x = n, no flow on the other sides."""
    rng = np.random.default_rng(seed)
    logk = rng.standard_normal((n, n))
    K = anisotropic_tensors(logk, rotation_2d(30.0), (1.0, 0.1))
    bc = {(0, 0): ("D", 1.0), (0, 1): ("D", 0.0)}
    indptr, indices, data, b = mpfa_o(K, bc)
    return dict(indptr=indptr, indices=indices, data=data, b=b, dims=(n, n), H=(H, H),
                centering=0, ncomp=1)


def darcy_3d_case(n=64, H=8, seed=1002, sigma=3.0, corr_len=8.0, dims=None):
    """3D MPFA-O case: ln k Gaussian random field (Gaussian covariance), tensor
    anisotropy 10:1 rotated by Euler angles (20, 35, 0) degrees, no-flow outer
    boundary, bottom-hole-pressure wells in two opposite corner cells."""
    dims = tuple(dims) if dims is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    logk = gaussian_random_field(dims, corr_len, sigma, rng)
    K = anisotropic_tensors(logk, rotation_zyx(20.0, 35.0, 0.0), (1.0, 1.0, 0.1))
    ncell = int(np.prod(dims))
    wells = [(0, 1.0), (ncell - 1, 0.0)]
    indptr, indices, data, b = mpfa_o(K, {}, wells)
    Hs = (H,) * 3 if np.isscalar(H) else tuple(H)
    return dict(indptr=indptr, indices=indices, data=data, b=b, dims=dims, H=Hs,
                centering=0, ncomp=1)


# ----------------------------------------------------------------------------
# MPFA-O on rough (perturbed) quadrilateral grids, 2D (Sec. 3.1 and 3.2)
# ----------------------------------------------------------------------------


def perturbed_grid(nx, ny, lx, ly, amp, rng, stretch_y=1.0):
    """Node coordinates (nx+1, ny+1) of a structured quadrilateral grid over
    [0, lx] x [0, ly*stretch_y]: interior nodes moved in x and y by amp * dx *
    psi, psi ~ U(-1/2, 1/2) (Sec. 3.2: amp = 0.2), boundary nodes fixed."""
    dx, dy = lx / nx, ly / ny
    X, Y = np.meshgrid(np.arange(nx + 1) * dx, np.arange(ny + 1) * dy, indexing="ij")
    px = amp * dx * (rng.uniform(size=X.shape) - 0.5)
    py = amp * dx * (rng.uniform(size=X.shape) - 0.5)
    inner = np.zeros(X.shape, dtype=bool)
    inner[1:-1, 1:-1] = True
    X = X + np.where(inner, px, 0.0)
    Y = (Y + np.where(inner, py, 0.0)) * stretch_y
    return X, Y


def mpfa_o_quads(X, Y, K, bc=None):
    """MPFA-O (continuity points at the edge midpoints) on a structured 2D
    quadrilateral grid with node coordinates X, Y (nx+1, ny+1) and cell
    tensors K (nx, ny, 2, 2); cells flat i + nx*j.

    In the interaction region of every node (up to four cells around it, four
    half-edges towards the neighbouring nodes) the pressure is linear in each
    cell, through the cell pressure at the cell centre (mean of its corners)
    and the potentials u_e at the midpoints of its two edges touching the node;
    the outward half-edge flux is -n^T K grad p with n the half-edge normal
    scaled by its length. Flux continuity on interior half-edges and the
    boundary condition on boundary ones (bc[(axis, side)] = ("D", value or
    f(x, y)) for Dirichlet, absent for no flow; axis 0: the x = min / max
    sides, axis 1: y) give a local system u = C^-1 (D p + e), which expresses
    every half-edge flux in the cell pressures.
    Returns (indptr, indices, data, b): int32 CSR (9-point stencil) and b."""
    bc = bc or {}
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    nx, ny = K.shape[:2]
    ncell = nx * ny
    xc = 0.25 * (X[:-1, :-1] + X[1:, :-1] + X[1:, 1:] + X[:-1, 1:])
    yc = 0.25 * (Y[:-1, :-1] + Y[1:, :-1] + Y[1:, 1:] + Y[:-1, 1:])
    I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    I, J = I.ravel(), J.ravel()
    nv = I.size
    xv, yv = X[I, J], Y[I, J]

    def node(di, dj):  # neighbour node coordinates (clipped where absent)
        ii, jj = np.clip(I + di, 0, nx), np.clip(J + dj, 0, ny)
        return X[ii, jj], Y[ii, jj], (I + di >= 0) & (I + di <= nx) & (J + dj >= 0) & (J + dj <= ny)

    # half-edges E, W, N, S: continuity point, normal from cell a to cell b
    hx, hy, hok, mid, nrm = [], [], [], [], []
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        x2, y2, ok = node(di, dj)
        mx, my = 0.5 * (xv + x2), 0.5 * (yv + y2)
        hxe, hye = mx - xv, my - yv
        mid.append((mx, my))
        hok.append(ok)
        if (di, dj) in ((1, 0), (0, -1)):  # left normal
            nrm.append((-hye, hxe))
        else:  # right normal
            nrm.append((hye, -hxe))
    # local cells SW, SE, NW, NE and their (a, b) roles on the half-edges
    cells = [(-1, -1), (0, -1), (-1, 0), (0, 0)]
    cid, cok = [], []
    for ci, cj in cells:
        ii, jj = I + ci, J + cj
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny)
        cok.append(ok)
        cid.append(np.where(ok, np.clip(ii, 0, nx - 1) + nx * np.clip(jj, 0, ny - 1), 0))
    # half-edge e: (cell a, cell b); E: SE|NE, W: SW|NW, N: NW|NE, S: SW|SE
    pair = [(1, 3), (0, 2), (2, 3), (0, 1)]
    # half-edges of each cell (in a fixed order)
    cedges = [(1, 3), (0, 3), (1, 2), (0, 2)]
    # w[c][e] (nv, 2): outward flux of cell c through its half-edge e in terms
    # of (u_e1 - p_c, u_e2 - p_c): -n^T K R^-1
    W = np.zeros((nv, 4, 4, 2))  # [vertex, cell, half-edge, k]
    for c in range(4):
        ci, cj = cells[c]
        ii, jj = np.clip(I + ci, 0, nx - 1), np.clip(J + cj, 0, ny - 1)
        Kc = K[ii, jj]
        xcc, ycc = xc[ii, jj], yc[ii, jj]
        e1, e2 = cedges[c]
        R = np.stack([np.stack([mid[e1][0] - xcc, mid[e1][1] - ycc], -1),
                      np.stack([mid[e2][0] - xcc, mid[e2][1] - ycc], -1)], 1)  # (nv, 2, 2)
        R[~cok[c]] = np.eye(2)
        Rinv = np.linalg.inv(R)
        for e in (e1, e2):
            sgn = 1.0 if pair[e][0] == c else -1.0
            n = sgn * np.stack(nrm[e], -1)  # (nv, 2) outward normal of c
            W[:, c, e] = -np.einsum("vi,vij,vjk->vk", n, Kc, Rinv)
    # local system C u = D p + ebc over the 4 half-edges
    C = np.zeros((nv, 4, 4))
    D = np.zeros((nv, 4, 4))
    ebc = np.zeros((nv, 4))
    flux_cells = []  # (e, c, mask) contributions to the cell balances
    for e in range(4):
        a, b = pair[e]
        pa, pb = cok[a], cok[b]
        both = pa & pb & hok[e]
        one = (pa ^ pb) & hok[e]
        absent = ~(both | one)
        # the boundary side of a one-sided half-edge
        if e in (0, 1):  # E, W: on y = min (cells above only) or y = max
            side_key = np.where(pb, 0, 1)  # only the upper cell b present -> bottom side
            axis = 1
        else:  # N, S: on x = min (only the right cell b) or x = max
            side_key = np.where(pb, 0, 1)
            axis = 0
        mx, my = mid[e]
        dir_mask = np.zeros(nv, dtype=bool)
        dval = np.zeros(nv)
        for side in (0, 1):
            kind = bc.get((axis, side))
            if kind is not None and kind[0] == "D":
                msk = one & (side_key == side)
                dir_mask |= msk
                v = kind[1](mx, my) if callable(kind[1]) else np.full(nv, float(kind[1]))
                dval = np.where(msk, v, dval)
        neu = one & ~dir_mask
        ident = absent | dir_mask
        # continuity: F_a + F_b = 0; Neumann: F_present = 0
        for c in (a, b):
            use = both | (neu & cok[c])
            e1, e2 = cedges[c]
            C[:, e, e1] += np.where(use, W[:, c, e, 0], 0.0)
            C[:, e, e2] += np.where(use, W[:, c, e, 1], 0.0)
            D[:, e, c] += np.where(use, W[:, c, e, 0] + W[:, c, e, 1], 0.0)
        C[:, e, e] += ident
        ebc[:, e] = np.where(dir_mask, dval, 0.0)
        for c in (a, b):
            flux_cells.append((e, c, cok[c] & (both | dir_mask)))
    Cinv = np.linalg.inv(C)
    Up = np.einsum("vij,vjk->vik", Cinv, D)  # u = Up p + ue
    ue = np.einsum("vij,vj->vi", Cinv, ebc)
    rows, cols, vals = [], [], []
    b = np.zeros(ncell)
    for e, c, msk in flux_cells:
        e1, e2 = cedges[c]
        w1, w2 = W[:, c, e, 0], W[:, c, e, 1]
        coef = w1[:, None] * Up[:, e1, :] + w2[:, None] * Up[:, e2, :]  # d F / d p_local
        coef[:, c] -= w1 + w2
        const = w1 * ue[:, e1] + w2 * ue[:, e2]
        for cc in range(4):
            m2 = msk & cok[cc]
            rows.append(cid[c][m2])
            cols.append(cid[cc][m2])
            vals.append(coef[m2, cc])
        np.add.at(b, cid[c][msk], -const[msk])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(ncell, ncell))
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64), b


def darcy_2d_perturbed_case(n=100, H=5, seed=1006, lx=20.0, ly=150.0, amp=0.2):
    """The 2D MPFA-O test of Sec. 3.2: an n x n grid on an lx x ly domain with
    interior nodes perturbed by amp * dx * U(-1/2, 1/2) in x and y, the tensor
    [[100, 25], [25, 100]] in every cell, unit pressure drop from x = 0 (p = 1)
    to x = lx (p = 0), no flow at the other sides, coarse blocks of H x H
    cells."""
    rng = np.random.default_rng(seed)
    X, Y = perturbed_grid(n, n, lx, ly, amp, rng)
    K = np.broadcast_to(np.array([[100.0, 25.0], [25.0, 100.0]]), (n, n, 2, 2)).copy()
    indptr, indices, data, b = mpfa_o_quads(X, Y, K, {(0, 0): ("D", 1.0), (0, 1): ("D", 0.0)})
    return dict(indptr=indptr, indices=indices, data=data, b=b, dims=(n, n), H=(H, H), centering=0, ncomp=1,
                X=X, Y=Y)
