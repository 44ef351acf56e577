"""Q1 (trilinear hexahedral) finite-element linear elasticity on unit cubes.

The stiffness matrix is returned in 3x3 block-CSR (BSR) over grid nodes with the
displacement components of a node interleaved (dof = 3*node + component); nodes
are ordered with x fastest. The isotropic elasticity tensor is
C = lambda I(x)I + 2G I4 with lambda = E nu / ((1+nu)(1-2nu)), G = E / (2(1+nu)),
so each element matrix is lambda_e * K_lambda + G_e * K_G with K_lambda, K_G
integrated once for the unit cube by 2x2x2 Gauss quadrature.
Fixed displacements are imposed by symmetric diagonalisation: the rows and
columns of the fixed dofs are zeroed except their diagonal entry, and the
right-hand side is updated (the fixed values here are zero).
"""
import itertools

import numpy as np

from .fields import gaussian_random_field

_LOCAL = [(ax, ay, az) for az in (0, 1) for ay in (0, 1) for ax in (0, 1)]


def _unit_cube_matrices():
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    Klam = np.zeros((24, 24))
    KG = np.zeros((24, 24))
    m = np.array([1.0, 1, 1, 0, 0, 0])
    Dlam = np.outer(m, m)
    DG = np.diag([2.0, 2, 2, 1, 1, 1])
    for xi in itertools.product(g, g, g):
        B = np.zeros((6, 24))
        for a, (ax, ay, az) in enumerate(_LOCAL):
            f = [xi[0] if ax else 1 - xi[0], xi[1] if ay else 1 - xi[1], xi[2] if az else 1 - xi[2]]
            s = [1.0 if ax else -1.0, 1.0 if ay else -1.0, 1.0 if az else -1.0]
            dN = np.array([s[0] * f[1] * f[2], s[1] * f[0] * f[2], s[2] * f[0] * f[1]])
            c = 3 * a
            B[0, c + 0] = dN[0]
            B[1, c + 1] = dN[1]
            B[2, c + 2] = dN[2]
            B[3, c + 1] = dN[2]
            B[3, c + 2] = dN[1]
            B[4, c + 0] = dN[2]
            B[4, c + 2] = dN[0]
            B[5, c + 0] = dN[1]
            B[5, c + 1] = dN[0]
        Klam += B.T @ Dlam @ B / 8.0
        KG += B.T @ DG @ B / 8.0
    return Klam, KG


def _offsets3():
    return [tuple(reversed(t)) for t in itertools.product((-1, 0, 1), repeat=3)]


def q1_elasticity(E, nu, fixed_bottom=True, top_traction=(0.0, 0.0, -1.0)):
    """Assemble K u = f on a grid of unit-cube elements.

    E, nu : arrays of shape (nex, ney, nez), per element.
    Returns dict(indptr, indices, data(nnzb,3,3), b(3*nnode), node_dims,
    fixed(bool per node)).
    """
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    ne = E.shape
    nn = tuple(s + 1 for s in ne)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    G = E / (2.0 * (1.0 + nu))
    Klam, KG = _unit_cube_matrices()
    offs = _offsets3()
    st = {o: k for k, o in enumerate(offs)}
    Ablk = np.zeros(nn + (27, 3, 3))
    esl = tuple(slice(0, s) for s in ne)
    for a, oa in enumerate(_LOCAL):
        nsl = tuple(slice(oa[d], oa[d] + ne[d]) for d in range(3))
        for b, ob in enumerate(_LOCAL):
            rel = tuple(ob[d] - oa[d] for d in range(3))
            blk_l = Klam[3 * a:3 * a + 3, 3 * b:3 * b + 3]
            blk_g = KG[3 * a:3 * a + 3, 3 * b:3 * b + 3]
            Ablk[nsl + (st[rel],)] += lam[esl][..., None, None] * blk_l + G[esl][..., None, None] * blk_g

    nnode = int(np.prod(nn))
    coords = np.indices(nn).reshape(3, -1, order="F")
    flat = np.arange(nnode)
    A_flat = np.moveaxis(Ablk, [0, 1, 2], [2, 1, 0]).reshape(nnode, 27, 3, 3)
    strides = [1, nn[0], nn[0] * nn[1]]
    fixed = (coords[2] == 0) if fixed_bottom else np.zeros(nnode, dtype=bool)

    f = np.zeros((nnode, 3))
    if top_traction is not None:
        # consistent load of a uniform traction on each unit top face: 1/4 per node
        cnt = np.zeros(nn[:2])
        cnt[:-1, :-1] += 1
        cnt[1:, :-1] += 1
        cnt[:-1, 1:] += 1
        cnt[1:, 1:] += 1
        top = coords[2] == nn[2] - 1
        w = cnt.reshape(-1, order="F") * 0.25
        f[top] += w[:, None] * np.asarray(top_traction)[None, :]

    rows, cols, vals = [], [], []
    for s, o in enumerate(offs):
        ok = np.ones(nnode, dtype=bool)
        shift = 0
        for d in range(3):
            c = coords[d] + o[d]
            ok &= (c >= 0) & (c < nn[d])
            shift += o[d] * strides[d]
        r = flat[ok]
        rows.append(r)
        cols.append(r + shift)
        vals.append(A_flat[ok, s])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order].copy()

    # symmetric diagonalisation of the fixed (zero) displacements
    fr = fixed[rows]
    fc = fixed[cols]
    diag_blk = rows == cols
    keep_diag = np.zeros_like(vals)
    keep_diag[:] = np.eye(3)[None] * vals
    vals[fr | fc] = 0.0
    vals[fr & diag_blk] = keep_diag[fr & diag_blk]
    f[fixed] = 0.0

    indptr = np.zeros(nnode + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return dict(indptr=indptr.astype(np.int32), indices=cols.astype(np.int32), data=vals,
                b=f.reshape(-1), node_dims=nn, fixed=fixed)


def elastic_3d_case(ne=48, H=6, seed=1003, corr_len=6.0):
    """Heterogeneous elastic block: ln E Gaussian random field around ln(1e10)
    with unit standard deviation, nu ~ U(0.2, 0.35) per element, bottom face
    fixed, unit downward traction on the top face."""
    rng = np.random.default_rng(seed)
    dims = (ne, ne, ne) if np.isscalar(ne) else tuple(ne)
    lnE = np.log(1e10) + gaussian_random_field(dims, corr_len, 1.0, rng)
    nu = rng.uniform(0.2, 0.35, size=dims)
    out = q1_elasticity(np.exp(lnE), nu)
    Hs = (H,) * 3 if np.isscalar(H) else tuple(H)
    out.update(dims=out["node_dims"], H=Hs, centering=1, ncomp=3)
    return out
