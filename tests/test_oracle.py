"""Pins of the FP64 oracle against what the paper and the mathematics fix
(hand-derived values, closed forms, invariants, brute force on tiny inputs)."""
from fractions import Fraction
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from oracle import msrsb as O
from synth.darcy import tpfa, mpfa_o, darcy_2d_case, darcy_3d_case, anisotropic_tensors
from synth.elastic import q1_elasticity, elastic_3d_case
from synth.fields import rotation_2d


def _csr(t):
    A = sp.csr_matrix((t[2], t[1], t[0]))
    A.sort_indices()
    return A


def _unit_tpfa(dims, bc=None):
    d = len(dims)
    K = np.zeros(dims + (d, d))
    for a in range(d):
        K[..., a, a] = 1.0
    return _csr(tpfa(K, bc or {}))


# ---------------- partition ----------------

@pytest.mark.parametrize("dims,H,cen", [((64, 64), (8, 8), 0), ((64, 64, 64), (8, 8, 8), 0),
                                        ((49, 49, 49), (6, 6, 6), 1), ((13, 9), (3, 4), 0)])
def test_partition_counts(dims, H, cen):
    part = O.partition(dims, H, cen)
    pat = part["pat"]
    d = len(dims)
    sizes = np.diff(pat.indptr)
    assert sizes.min() >= 1 and sizes.max() <= 2 ** d
    # skeleton rows are exactly those in fewer than 2^d supports, unless a
    # domain edge cuts the support (rows before the first / after the last node)
    assert np.all(sizes[~part["skel"]] >= 1)
    # closed-form nnz: per axis, points with one id count 1, with two count 2
    expect = 1
    for a in range(d):
        c, _ = O.coarse_axis(dims[a], H[a], cen)
        x = np.arange(dims[a])
        two = (x > c[0]) & (x < c[-1]) & ~np.isin(x, c)
        expect *= int((~two).sum() + 2 * two.sum())
    assert pat.nnz == expect
    # every point's primal block is among its pattern ids (block within support)
    rows = np.repeat(np.arange(pat.shape[0]), sizes)
    hit = np.zeros(pat.shape[0], bool)
    hit[rows[pat.indices == part["part"][rows]]] = True
    assert hit.all()
    # coarse node of J lies in block J and on the skeleton
    assert np.all(part["part"][part["cnode"]] == np.arange(part["nc"]))
    assert part["skel"][part["cnode"]].all()


def test_partition_paper_sizes():
    assert O.partition((64, 64), (8, 8), 0)["pat"].nnz == 113 ** 2
    assert O.partition((49, 49, 49), (6, 6, 6), 1)["pat"].nnz == 89 ** 3
    _, blk = O.coarse_axis(49, 6, 1)
    assert list(np.bincount(blk)) == [4, 6, 6, 6, 6, 6, 6, 6, 3]


def test_partition_bruteforce_supports():
    # supports by direct definition: open interval between neighbouring nodes
    dims, H = (10, 7), (4, 3)
    part = O.partition(dims, H, 0)
    cx, _ = O.coarse_axis(10, 4, 0)
    cy, _ = O.coarse_axis(7, 3, 0)
    pat = part["pat"].toarray() > 0
    for x in range(10):
        for y in range(7):
            for Ix in range(len(cx)):
                for Iy in range(len(cy)):
                    inx = (Ix == 0 or x > cx[Ix - 1]) and (Ix == len(cx) - 1 or x < cx[Ix + 1])
                    iny = (Iy == 0 or y > cy[Iy - 1]) and (Iy == len(cy) - 1 or y < cy[Iy + 1])
                    assert pat[x + 10 * y, Ix + len(cx) * Iy] == (inx and iny)


# ---------------- filter ----------------

def test_filter_invariants_mpfa():
    c = darcy_2d_case(n=16)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    Ah = O.mmatrix_filter(A)
    off = Ah - sp.diags(Ah.diagonal())
    assert off.data.max() <= 0.0
    scale = np.asarray(abs(A).sum(axis=1)).ravel()
    assert np.all(np.abs(np.asarray(Ah.sum(axis=1)).ravel()) <= 1e-15 * scale * 4)
    # positive off-diagonals removed, negative ones kept verbatim
    Ad, Ahd = A.toarray(), Ah.toarray()
    m = ~np.eye(A.shape[0], dtype=bool)
    assert np.array_equal(Ahd[m], np.minimum(Ad[m], 0.0))
    # diagonal ignores A's own diagonal (wells / Dirichlet terms have no effect)
    assert np.allclose(np.diag(Ahd), -np.minimum(Ad * m, 0).sum(axis=1), rtol=1e-15, atol=0)


def test_filter_noop_on_mmatrix_offdiagonals():
    A = _unit_tpfa((6, 5), {(0, 0): ("D", 1.0)})
    Ah = O.mmatrix_filter(A)
    assert np.array_equal((Ah - sp.diags(Ah.diagonal())).toarray(), (A - sp.diags(A.diagonal())).toarray())


def test_sdc_blocks():
    rng = np.random.default_rng(0)
    e = q1_elasticity(np.exp(rng.standard_normal((2, 2, 2))), rng.uniform(0.2, 0.35, (2, 2, 2)))
    comps = O.sdc_blocks(e["indptr"], e["indices"], e["data"])
    full = O.bsr_to_csr(e["indptr"], e["indices"], e["data"]).toarray()
    for l in range(3):
        assert np.array_equal(comps[l].toarray(), full[l::3, l::3])


# ---------------- basis ----------------

def _load_first_step(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "basis_first_step_9x3_H3.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            x, y, J, num, den = map(int, line.split())
            rows.append((x, y, J, Fraction(num, den)))
    return rows


def test_basis_first_pass_hand_values(golden_dir):
    dims, H = (9, 3), (3, 3)
    A = _unit_tpfa(dims)
    part = O.partition(dims, H, 0)
    P0 = O.indicator(part["part"], part["pat"])
    vals, k, e_it, hist = O.enhanced_msrsb(O.mmatrix_filter(A), part["pat"], P0, part["skel"],
                                           tol=0.0, n_it=1, max_iter=1)
    Pm = O.as_matrix(vals, part["pat"]).toarray()
    for x, y, J, v in _load_first_step(golden_dir):
        assert abs(Pm[x + 9 * y, J] - float(v)) < 1e-15, (x, y, J)
    assert k == 1 and abs(e_it - 2.0 / 9.0) < 1e-15


def _hats(n, H, cen):
    c, _ = O.coarse_axis(n, H, cen)
    M = np.zeros((n, len(c)))
    for I in range(len(c)):
        for x in range(n):
            if I > 0 and c[I - 1] < x <= c[I]:
                M[x, I] = (x - c[I - 1]) / (c[I] - c[I - 1])
            elif I + 1 < len(c) and c[I] <= x < c[I + 1]:
                M[x, I] = (c[I + 1] - x) / (c[I + 1] - c[I])
            elif (I == 0 and x <= c[0]) or (I == len(c) - 1 and x >= c[-1]):
                M[x, I] = 1.0
    return M


@pytest.mark.parametrize("dims,H", [((16, 12), (4, 4)), ((13, 9), (3, 3)), ((9, 10, 7), (3, 4, 3))])
def test_basis_fixed_point_is_tensor_hats(dims, H):
    # reflection-symmetric zero-row-sum stencil: the converged basis is the
    # tensor product of 1D piecewise-linear hats through the coarse nodes
    # (the "bilinear interpolators" of Sec. 4, Fig. 7d)
    A = _unit_tpfa(dims)
    part = O.partition(dims, H, 0)
    P0 = O.indicator(part["part"], part["pat"])
    vals, k, e_it, _ = O.enhanced_msrsb(O.mmatrix_filter(A), part["pat"], P0, part["skel"],
                                        tol=1e-13, n_it=1, max_iter=20000)
    full = _hats(dims[0], H[0], 0)
    for a in range(1, len(dims)):
        full = np.kron(_hats(dims[a], H[a], 0), full)
    assert e_it <= 1e-13
    assert np.abs(O.as_matrix(vals, part["pat"]).toarray() - full).max() < 1e-10


def test_basis_fe_homogeneous_recovers_trilinear():
    # the paper's FE demo (Sec. 4, Fig. 7d): on a homogeneous Cartesian FE mesh
    # the filtered SDC component recovers (bi/tri)linear interpolators. The Q1
    # stencil of one displacement component is reflection symmetric, so the
    # fixed point is the tensor product of 1D hats through the coarse nodes.
    e = q1_elasticity(np.ones((9, 6, 3)), 0.25 * np.ones((9, 6, 3)), fixed_bottom=False, top_traction=None)
    comps = O.sdc_blocks(e["indptr"], e["indices"], e["data"])
    dims = e["node_dims"]
    part = O.partition(dims, (3, 3, 3), 1)
    P0 = O.indicator(part["part"], part["pat"])
    for l in range(3):
        vals, k, e_it, _ = O.enhanced_msrsb(O.mmatrix_filter(comps[l]), part["pat"], P0, part["skel"],
                                            tol=1e-12, n_it=1, max_iter=20000)
        full = np.kron(_hats(4, 3, 1), np.kron(_hats(7, 3, 1), _hats(10, 3, 1)))
        assert k > 10 and e_it <= 1e-12
        assert np.abs(O.as_matrix(vals, part["pat"]).toarray() - full).max() < 1e-9


def test_basis_invariants_mpfa():
    c = darcy_3d_case(n=16)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    part = O.partition(c["dims"], c["H"], 0)
    P0 = O.indicator(part["part"], part["pat"])
    vals, k, e_it, hist = O.enhanced_msrsb(O.mmatrix_filter(A), part["pat"], P0, part["skel"],
                                           tol=0.0, n_it=10, max_iter=50)
    P = O.as_matrix(vals, part["pat"])
    assert np.abs(np.asarray(P.sum(axis=1)).ravel() - 1.0).max() < 1e-14
    assert vals.min() >= 0.0 and vals.max() <= 1.0 + 1e-15
    assert k == 50 and [h[0] for h in hist] == [0, 10, 20, 30, 40]
    # e_it decreases between checks on the filtered operator
    es = [h[1] for h in hist]
    assert all(b < a for a, b in zip(es, es[1:]))


def test_unfiltered_basis_leaves_unit_interval():
    # Sec. 3.1 / Fig. 3c: smoothing with the unfiltered MPFA-O operator loses
    # monotonicity (entries leave [0, 1]); the filtered operator keeps them.
    # strong rotated anisotropy (1000:1 at 30 degrees) stands in for the
    # paper's perturbed, 10x stretched grid: both make MPFA-O far from an M-matrix
    n = 16
    K = anisotropic_tensors(np.zeros((n, n)), rotation_2d(30.0), (1.0, 0.001))
    A = _csr(mpfa_o(K, {}))
    part = O.partition((n, n), (4, 4), 0)
    P0 = O.indicator(part["part"], part["pat"])
    Ah = A.copy()
    Ah.setdiag(0)
    Ah.eliminate_zeros()
    Ah = (Ah - sp.diags(np.asarray(Ah.sum(axis=1)).ravel())).tocsr()  # zero row sum, not filtered
    raw, *_ = O.enhanced_msrsb(Ah, part["pat"], P0, part["skel"], tol=0.0, max_iter=30)
    filt, *_ = O.enhanced_msrsb(O.mmatrix_filter(A), part["pat"], P0, part["skel"], tol=0.0, max_iter=30)
    assert raw.min() < -1e-2 or raw.max() > 1 + 1e-2
    assert filt.min() >= 0 and filt.max() <= 1 + 1e-15


# ---------------- Galerkin ----------------

def test_galerkin_identity_prolongation():
    c = darcy_3d_case(n=6)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    part = O.partition(c["dims"], (1, 1, 1), 0)
    P = O.as_matrix(O.indicator(part["part"], part["pat"]), part["pat"])
    assert np.array_equal(O.galerkin(A, P).toarray(), A.toarray())


def test_galerkin_rowsums_and_dense():
    c = darcy_3d_case(n=12, H=4)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    s = O.setup_scalar(A, c["dims"], c["H"], tol=0.0, max_iter=10)
    P = s["P"]
    Ac = s["tl"].Ac.toarray()
    Pd, Ad = P.toarray(), A.toarray()
    dense = Pd.T @ Ad @ Pd
    assert np.abs(Ac - dense).max() <= 1e-12 * np.abs(dense).max()
    # partition of unity: A_c 1 = P^T (A 1); A has wells, so A 1 != 0 and a
    # Galerkin product built from the filtered operator would fail this
    lhs = Ac @ np.ones(Ac.shape[0])
    rhs = Pd.T @ (Ad @ np.ones(A.shape[0]))
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(Ac).max()
    assert np.abs(rhs).max() > 1e-3 * np.abs(Ac).max()


def test_galerkin_symmetric_spd_elastic():
    rng = np.random.default_rng(1)
    e = q1_elasticity(np.exp(rng.standard_normal((6, 6, 6))), rng.uniform(0.2, 0.35, (6, 6, 6)))
    s = O.setup_elastic(e["indptr"], e["indices"], e["data"], e["node_dims"], (3, 3, 3), tol=0.0, max_iter=5)
    Ac = s["tl"].Ac.toarray()
    assert np.abs(Ac - Ac.T).max() <= 1e-13 * np.abs(Ac).max()
    assert np.linalg.eigvalsh(Ac).min() > 0


# ---------------- smoothers ----------------

def test_parity_colouring_is_valid():
    c = darcy_3d_case(n=6)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    col = O.parity_colours(c["dims"])
    r = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    off = r != A.indices
    assert np.all(col[r[off]] != col[A.indices[off]])
    assert col.max() == 7


@pytest.mark.parametrize("order", ["colour", "natural", "lines"])
def test_ilu0_defining_property(order):
    """(L U)_ij = A_ij on A's pattern, in every elimination order."""
    c = darcy_3d_case(dims=(8, 7, 5))
    A = _csr((c["indptr"], c["indices"], c["data"]))
    if order == "lines":
        lo, lcol, _, _ = O.line_block_order(c["dims"])
        sm = O.ColouredSmoother(A, lcol, "ilu0", order=lo)
    else:
        sm = O.ColouredSmoother(A, O.parity_colours(c["dims"]) if order == "colour" else None, "ilu0")
    if order == "natural":
        assert np.array_equal(sm.order, np.arange(A.shape[0]))
    B = sm.B
    L, U = sm.L, sm.U
    LU = ((L + sp.eye(B.shape[0])) @ U).toarray()
    mask = B.toarray() != 0
    mask |= np.eye(B.shape[0], dtype=bool)
    Bd = B.toarray()
    assert np.abs(LU[mask] - Bd[mask]).max() <= 1e-12 * np.abs(Bd).max()
    # the smoother inverts exactly its own factors: L U (M^-1 v) = v
    v = np.random.default_rng(3).standard_normal(A.shape[0])
    zp = sm.solve(v)[sm.order]
    assert np.abs((L + sp.eye(B.shape[0])) @ (U @ zp) - v[sm.order]).max() < 1e-11 * np.abs(v).max()


@pytest.mark.parametrize("dims", [(9, 7, 5), (6, 5), (5, 4, 4)])
def test_line_block_order_structure(dims):
    """The line-block order: blocks of one colour never share a 3^d stencil
    (each colour stage is independent across blocks), and inside a block a
    point's earlier neighbours are the previous point of its own x-line
    (sub-line) or points of the block's earlier sub-lines: the structure the
    GPU sweep relies on (a recurrence along x per sub-line)."""
    c = darcy_3d_case(dims=dims) if len(dims) == 3 else darcy_2d_case(n=dims[0], H=2)
    if len(dims) == 2:
        dims = c["dims"]
    A = _csr((c["indptr"], c["indices"], c["data"])).tocoo()
    order, colour, block, sub = O.line_block_order(dims)
    n = A.shape[0]
    assert np.array_equal(np.sort(order), np.arange(n))
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    x = np.arange(n) % dims[0]
    off = A.row != A.col
    r, k = A.row[off], A.col[off]
    same_colour = colour[r] == colour[k]
    assert np.all(block[r][same_colour] == block[k][same_colour])  # same colour: same block only
    earlier_in_block = (block[r] == block[k]) & (pos[k] < pos[r])
    rec = earlier_in_block & (sub[r] == sub[k])
    assert np.all(x[k][rec] == x[r][rec] - 1)
    assert np.all(sub[k][earlier_in_block & ~rec] < sub[r][earlier_in_block & ~rec])
    ncol = 2 ** (len(dims) - 1)
    assert colour.max() == ncol - 1


def test_ilu0_exact_for_tridiagonal():
    n = 40
    rng = np.random.default_rng(2)
    T = sp.diags([-rng.uniform(0.5, 1, n - 1), 3 + rng.uniform(0, 1, n), -rng.uniform(0.5, 1, n - 1)],
                 [-1, 0, 1], format="csr")
    L, U = O.ilu0(T)
    assert np.abs(((L + sp.eye(n)) @ U - T).toarray()).max() < 1e-14
    v = rng.standard_normal(n)
    # natural order on a chain: no fill, so ILU(0) is the exact LU and the
    # smoother is T^-1
    nat = O.ColouredSmoother(T, None, "ilu0")
    assert np.abs(T @ nat.solve(v) - v).max() < 1e-13
    sm = O.ColouredSmoother(T, np.zeros(n, dtype=np.int64) + (np.arange(n) % 2), "ilu0")
    # red-black order on a chain drops fill, so it is not exact; check that
    # the triangular solves satisfy L U z = v in that order
    z = sm.solve(v)
    B = sm.B
    Lp, Up = O.ilu0(B)
    zp = z[sm.order]
    assert np.abs(((Lp + sp.eye(n)) @ (Up @ zp)) - v[sm.order]).max() < 1e-13
    assert np.abs(T @ z - v).max() > 1e-6


@pytest.mark.parametrize("order", ["colour", "natural"])
def test_block_gauss_seidel_solves_its_triangle(order):
    rng = np.random.default_rng(4)
    e = q1_elasticity(np.exp(rng.standard_normal((3, 3, 3))), rng.uniform(0.2, 0.35, (3, 3, 3)))
    A = O.bsr_to_csr(e["indptr"], e["indices"], e["data"])
    col = O.parity_colours(e["node_dims"]) if order == "colour" else None
    v = rng.standard_normal(A.shape[0])
    for kind in ("gs_fwd", "gs_bwd"):
        sm = O.ColouredSmoother(A, col, kind, bdim=3)
        z = sm.solve(v)[sm.order]
        B = sm.B.toarray()
        node = np.arange(B.shape[0]) // 3
        keep = (node[:, None] == node[None, :])
        keep |= (np.arange(B.shape[0])[:, None] > np.arange(B.shape[0])[None, :]) if kind == "gs_fwd" else \
            (np.arange(B.shape[0])[:, None] < np.arange(B.shape[0])[None, :])
        M = np.where(keep, B, 0.0)
        assert np.abs(M @ z - v[sm.order]).max() < 1e-10 * np.abs(v).max()


@pytest.mark.parametrize("order", ["colour", "natural"])
def test_ic0_factors_are_symmetric_and_match_a_on_the_pattern(order):
    """IC(0) (Sec. 4.1, 4.3) as ILU(0) of the SPD elasticity operator in node
    order: L U = A on A's pattern and U = diag(U) L^T, i.e. M = L D L^T."""
    rng = np.random.default_rng(14)
    e = q1_elasticity(np.exp(rng.standard_normal((3, 3, 3))), rng.uniform(0.2, 0.35, (3, 3, 3)))
    A = O.bsr_to_csr(e["indptr"], e["indices"], e["data"])
    sm = O.ColouredSmoother(A, O.parity_colours(e["node_dims"]) if order == "colour" else None, "ilu0", bdim=3)
    B = sm.B.toarray()
    L = sm.L.toarray() + np.eye(B.shape[0])
    U = sm.U.toarray()
    mask = B != 0
    assert np.abs((L @ U)[mask] - B[mask]).max() <= 1e-12 * np.abs(B).max()
    assert np.abs(U - np.diag(np.diag(U)) @ L.T).max() <= 1e-12 * np.abs(U).max()
    assert np.diag(U).min() > 0


def test_ic0_is_exact_on_a_chain_of_blocks():
    """On a block-tridiagonal SPD matrix (a chain of nodes with 3x3 blocks)
    the natural-order IC(0) drops no fill, so M = A; the parity order (red-
    black nodes) drops fill and is not exact."""
    rng = np.random.default_rng(15)
    nn = 12
    blocks = []
    rows = []
    cols = []
    for i in range(nn):
        for j in (i - 1, i, i + 1):
            if 0 <= j < nn:
                rows.append(i)
                cols.append(j)
    off = {}
    for i in range(nn - 1):
        off[i] = -rng.uniform(0.2, 0.5, (3, 3))
    data = []
    for i, j in zip(rows, cols):
        if i == j:
            data.append(np.eye(3) * 4 + 0.1 * np.ones((3, 3)))
        elif j == i + 1:
            data.append(off[i])
        else:
            data.append(off[j].T)
    indptr = np.searchsorted(rows, np.arange(nn + 1))
    A = O.bsr_to_csr(indptr, np.array(cols), np.array(data))
    assert np.linalg.eigvalsh(A.toarray()).min() > 0
    v = rng.standard_normal(3 * nn)
    nat = O.ColouredSmoother(A, None, "ilu0", bdim=3)
    assert np.abs(A @ nat.solve(v) - v).max() <= 1e-12 * np.abs(v).max()
    rb = O.ColouredSmoother(A, np.arange(nn) % 2, "ilu0", bdim=3)
    assert np.abs(A @ rb.solve(v) - v).max() > 1e-6


def test_ic0_two_stage_operator_is_symmetric():
    """IC(0) before and after the coarse stage gives a symmetric two-stage
    operator, as PCG needs (Sec. 4)."""
    rng = np.random.default_rng(16)
    e = q1_elasticity(np.exp(rng.standard_normal((4, 3, 3))), rng.uniform(0.2, 0.35, (4, 3, 3)))
    s = O.setup_elastic(e["indptr"], e["indices"], e["data"], e["node_dims"], (2, 2, 2), tol=0.0, max_iter=8,
                        smoother="ic0")
    n = s["A"].shape[0]
    I = np.eye(n)
    Minv = np.column_stack([s["tl"].apply(I[:, j]) for j in range(n)])
    assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0


def test_block_prolongation_interleaves_components():
    """Sec. 4: component l of every fine node is interpolated from component l
    of the coarse nodes only, with that component's own basis. Three different
    bases on one pattern (the block indicator, a smoothed basis, random
    row-normalised values): column 3J+l of P is basis l of coarse node J on
    rows 3i+l and zero on the other components, and the rows of each
    component block sum to the identity (sum_J P[3i+l, 3J+m] = delta_lm)."""
    dims, H = (5, 5, 5), (2, 2, 2)
    part = O.partition(dims, H, 1)
    pat, nc = part["pat"], part["nc"]
    n = pat.shape[0]
    rng = np.random.default_rng(12)
    b0 = O.indicator(part["part"], pat)
    Ah = O.mmatrix_filter(_unit_tpfa(dims))
    b1 = O.enhanced_msrsb(Ah, pat, b0, part["skel"], tol=0.0, max_iter=7)[0]
    r = rng.uniform(0.1, 1.0, pat.nnz)
    rows = np.repeat(np.arange(n), np.diff(pat.indptr))
    b2 = r / np.bincount(rows, weights=r)[rows]
    Ps = [O.as_matrix(b, pat) for b in (b0, b1, b2)]
    assert not np.allclose(b0, b1) and not np.allclose(b1, b2)
    Pb = O.block_prolongation(Ps)
    assert Pb.shape == (3 * n, 3 * nc)
    dense = [P.toarray() for P in Ps]
    for J in range(nc):
        for l in range(3):
            e = np.zeros(3 * nc)
            e[3 * J + l] = 1.0
            col = (Pb @ e).reshape(n, 3)
            assert np.array_equal(col[:, l], dense[l][:, J])
            assert not col[:, [m for m in range(3) if m != l]].any()
    for m in range(3):
        ones_m = np.zeros(3 * nc)
        ones_m[m::3] = 1.0
        s = (Pb @ ones_m).reshape(n, 3)
        for l in range(3):
            assert np.abs(s[:, l] - (1.0 if l == m else 0.0)).max() <= 1e-14


# ---------------- two-stage apply ----------------

def test_two_level_matches_error_propagation_matrix():
    rng = np.random.default_rng(6)
    e = q1_elasticity(np.exp(rng.standard_normal((4, 3, 3))), rng.uniform(0.2, 0.35, (4, 3, 3)))
    s = O.setup_elastic(e["indptr"], e["indices"], e["data"], e["node_dims"], (2, 2, 2), tol=0.0, max_iter=8)
    tl = s["tl"]
    A = tl.A.toarray()
    n = A.shape[0]
    I = np.eye(n)
    Minv = np.column_stack([tl.apply(I[:, j]) for j in range(n)])
    Mpre = np.column_stack([tl.pre.solve(I[:, j]) for j in range(n)])
    Mpost = np.column_stack([tl.post.solve(I[:, j]) for j in range(n)])
    P = tl.P.toarray()
    C = P @ np.linalg.solve(P.T @ A @ P, P.T)
    E = (I - Mpost @ A) @ (I - C @ A) @ (I - Mpre @ A)
    ref = (I - E) @ np.linalg.inv(A)
    assert np.abs(Minv - ref).max() <= 1e-8 * np.abs(ref).max()
    # forward pre / backward post Gauss-Seidel make the preconditioner symmetric
    assert np.abs(Minv - Minv.T).max() <= 1e-8 * np.abs(Minv).max()


def test_coarse_correction_galerkin_orthogonality():
    c = darcy_2d_case(n=24)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    s = O.setup_scalar(A, c["dims"], c["H"], tol=0.0, max_iter=20)
    tl = s["tl"]
    v = np.random.default_rng(7).standard_normal(A.shape[0])
    r = v - A @ tl.multiscale(v)
    assert np.abs(tl.R @ r).max() <= 1e-10 * np.abs(tl.R @ v).max()
    w = np.random.default_rng(8).standard_normal(A.shape[0])
    assert np.allclose(tl.apply(2 * v - 3 * w), 2 * tl.apply(v) - 3 * tl.apply(w), rtol=0, atol=1e-10)


def test_fv_restriction_is_the_block_indicator():
    """Petrov-Galerkin R of Sec. 2 (the MSFV choice): row J sums the fine
    equations of primal block J; checked against blocks from cell coordinates
    (cell x lies in block x // H per axis) and, for 3x3 blocks, per component."""
    dims, H = (10, 7, 5), (4, 4, 2)
    part = O.partition(dims, H, 0)
    coords = np.indices(dims).reshape(3, -1, order="F")
    nb = [-(-d // h) for d, h in zip(dims, H)]
    blk = coords[0] // H[0] + nb[0] * (coords[1] // H[1] + nb[1] * (coords[2] // H[2]))
    R = O.fv_restriction(part["part"], part["nc"]).toarray()
    assert R.shape == (part["nc"], coords.shape[1])
    assert np.array_equal(R, (blk[None, :] == np.arange(part["nc"])[:, None]).astype(float))
    R3 = O.fv_restriction(part["part"], part["nc"], bdim=3).toarray()
    for l in range(3):
        assert np.array_equal(R3[l::3, l::3], R)
        for m in range(3):
            if m != l:
                assert not R3[l::3, m::3].any()


def test_fv_restriction_conserves_mass_on_every_coarse_block():
    """The finite-volume restriction makes the coarse correction conservative
    (Sec. 2): the residual v - A P A_c^-1 R v sums to zero over every primal
    block, while the Galerkin choice (R = P^T) does not give this."""
    c = darcy_2d_case(n=24)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    fv = O.setup_scalar(A, c["dims"], c["H"], tol=0.0, max_iter=20, restriction="fv")
    ga = O.setup_scalar(A, c["dims"], c["H"], tol=0.0, max_iter=20)
    v = np.random.default_rng(17).standard_normal(A.shape[0])
    Rb = O.fv_restriction(fv["part"]["part"], fv["part"]["nc"])
    r_fv = v - A @ fv["tl"].multiscale(v)
    r_ga = v - A @ ga["tl"].multiscale(v)
    assert np.abs(Rb @ r_fv).max() <= 1e-10 * np.abs(Rb @ v).max()
    assert np.abs(Rb @ r_ga).max() > 1e-6 * np.abs(Rb @ v).max()
    # A_c = R A P with P's rows summing to one: A_c 1 = R (A 1)
    Ac = fv["tl"].Ac
    assert np.abs(Ac @ np.ones(Ac.shape[0]) - Rb @ (A @ np.ones(A.shape[0]))).max() <= 1e-12 * abs(Ac).max()


def test_two_level_fv_matches_error_propagation_matrix():
    """Alg. 4 with the Petrov-Galerkin restriction equals (I - E) A^-1 with
    E = (I - M_post^-1 A)(I - P A_c^-1 R A), A_c = R A P, on a dense case."""
    c = darcy_2d_case(n=12, H=4)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    s = O.setup_scalar(A, c["dims"], c["H"], tol=0.0, max_iter=10, restriction="fv")
    tl = s["tl"]
    Ad = A.toarray()
    n = Ad.shape[0]
    I = np.eye(n)
    Minv = np.column_stack([tl.apply(I[:, j]) for j in range(n)])
    Mpost = np.column_stack([tl.post.solve(I[:, j]) for j in range(n)])
    P = tl.P.toarray()
    R = O.fv_restriction(s["part"]["part"], s["part"]["nc"]).toarray()
    C = P @ np.linalg.solve(R @ Ad @ P, R)
    E = (I - Mpost @ Ad) @ (I - C @ Ad)
    ref = (I - E) @ np.linalg.inv(Ad)
    assert np.abs(Minv - ref).max() <= 1e-8 * np.abs(ref).max()


# ---------------- Krylov ----------------

def test_gmres_matches_direct_solve():
    c = darcy_2d_case(n=32, H=8)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    s = O.setup_scalar(A, c["dims"], c["H"])
    x, its, rr, hist = O.gmres_right(A, c["b"], s["tl"].apply, rtol=1e-10)
    xs = np.linalg.solve(A.toarray(), c["b"])
    assert rr <= 1e-10
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)
    # the two-level preconditioner needs fewer iterations than its smoother
    _, its_s, _, _ = O.gmres_right(A, c["b"], s["tl"].post.solve, rtol=1e-10)
    assert its < its_s


def test_gmres_exact_preconditioner_one_iteration():
    c = darcy_2d_case(n=8)
    A = _csr((c["indptr"], c["indices"], c["data"]))
    s = O.setup_scalar(A, c["dims"], (1, 1), smoother=None)
    x, its, rr, _ = O.gmres_right(A, c["b"], s["tl"].apply)
    assert its == 1 and rr < 1e-12


def test_pcg_matches_direct_solve():
    rng = np.random.default_rng(9)
    e = q1_elasticity(np.exp(rng.standard_normal((6, 6, 6))), rng.uniform(0.2, 0.35, (6, 6, 6)))
    s = O.setup_elastic(e["indptr"], e["indices"], e["data"], e["node_dims"], (3, 3, 3), tol=1e-3)
    A = s["A"]
    x, its, rr, _ = O.pcg(A, e["b"], s["tl"].apply, rtol=1e-10)
    xs = np.linalg.solve(A.toarray(), e["b"])
    assert rr <= 1e-10
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)


# ---------------- l1-Jacobi smoother, smoothing-only baseline, Richardson ----------------

def test_l1_jacobi_exact_on_a_diagonal_matrix():
    d = np.array([2.0, 5.0, 0.5, 3.0])
    A = sp.diags(d).tocsr()
    r = np.array([1.0, -2.0, 3.0, 0.25])
    for sweeps in (1, 2, 3):
        assert np.allclose(O.L1Jacobi(A, sweeps).solve(r), r / d, rtol=0, atol=1e-15)


def test_l1_jacobi_two_sweeps_hand_values():
    # tridiag(-1, 2, -1), n = 5: d = (3, 4, 4, 4, 3); r = e_2 (0-based). Sweep 1:
    # z = (0, 0, 1/4, 0, 0); r - A z = (0, 1/4, 1/2, 1/4, 0); sweep 2 adds that / d.
    A = sp.diags([-np.ones(4), 2 * np.ones(5), -np.ones(4)], [-1, 0, 1]).tocsr()
    r = np.zeros(5)
    r[2] = 1.0
    z = O.L1Jacobi(A, 2).solve(r)
    assert np.allclose(z, [0.0, 1 / 16, 3 / 8, 1 / 16, 0.0], rtol=0, atol=1e-15)


def test_l1_jacobi_two_stage_operator_is_symmetric():
    c = elastic_3d_case(ne=4, H=2)
    st = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], tol=0.0, max_iter=10,
                         smoother="l1jac", sweeps=2)
    rng = np.random.default_rng(2)
    n = st["A"].shape[0]
    v, w = rng.standard_normal(n), rng.standard_normal(n)
    a, b = v @ st["tl"].apply(w), w @ st["tl"].apply(v)
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
    # and PCG with it converges to a dense solve
    x, its, rr, _ = O.pcg(st["A"], c["b"], st["tl"].apply, rtol=1e-10, maxit=300)
    xd = np.linalg.solve(st["A"].toarray(), c["b"])
    assert rr <= 1e-10 and np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_richardson_exact_preconditioner_one_step():
    A = sp.diags([-np.ones(9), 3 * np.ones(10), -np.ones(9)], [-1, 0, 1]).tocsc()
    b = np.arange(10.0)
    solve = sla.splu(A).solve
    x, its, rr, _ = O.richardson(A, b, solve, rtol=1e-12, maxit=5)
    assert its == 1 and rr <= 1e-14


def test_richardson_multiscale_vs_smoothing_only():
    # Sec. 3.2: MsRSB + ILU(0) as a stand-alone Richardson iteration converges,
    # ILU(0) alone does not within 150 iterations
    c = darcy_2d_case()
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    ms = O.setup_scalar(A, c["dims"], c["H"], tol=1e-3, max_iter=100)
    so = O.setup_scalar(A, c["dims"], c["H"], tol=1e-3, max_iter=100, coarse=False)
    _, its_ms, rr_ms, _ = O.richardson(A, c["b"], ms["tl"].apply, rtol=1e-8, maxit=150)
    _, its_so, rr_so, _ = O.richardson(A, c["b"], so["tl"].apply, rtol=1e-8, maxit=150)
    assert rr_ms <= 1e-8 and its_ms < 150
    assert rr_so > 1e-8


# ---------------- adjoint gradient of a TPFA objective ----------------

def test_adjoint_gradient_matches_brute_force_differences():
    # every cell of a 4 x 3 x 2 grid, central differences of J itself
    dims = (4, 3, 2)
    n = 24
    rng = np.random.default_rng(4)
    logk = rng.standard_normal(n)
    obs = np.array([1, 7, 13, 22])
    p_obs = rng.uniform(0.2, 0.8, size=4)
    J, g, _ = O.tpfa_objective_gradient(dims, logk, obs, p_obs)
    eps = 1e-5
    fd = np.empty(n)
    for c in range(n):
        e = np.zeros(n)
        e[c] = eps
        fd[c] = (O.tpfa_objective_gradient(dims, logk + e, obs, p_obs)[0]
                 - O.tpfa_objective_gradient(dims, logk - e, obs, p_obs)[0]) / (2 * eps)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(fd).max()


def test_adjoint_gradient_zero_at_the_observed_field():
    # p_obs equal to the model's own pressures: J = 0 and dJ/dtheta = 0
    dims = (5, 4)
    rng = np.random.default_rng(5)
    logk = rng.standard_normal(20)
    obs = np.array([2, 9, 17])
    _, _, p = O.tpfa_objective_gradient(dims, logk, obs, np.zeros(3))
    J, g, _ = O.tpfa_objective_gradient(dims, logk, obs, p[obs])
    assert J <= 1e-28 and np.abs(g).max() <= 1e-14


def _mpfa_J(K_hat, logk, wells, obs, p_obs):
    from synth.darcy import mpfa_o
    dims = K_hat.shape[:3]
    K = np.exp(logk).reshape(dims, order="F")[..., None, None] * K_hat
    ip, ix, d, b = mpfa_o(K, {}, wells)
    A = sp.csr_matrix((d, ix, ip))
    p = sla.spsolve(A.tocsc(), b)
    return float(((p[obs] - p_obs) ** 2).sum()), A, b


def test_mpfa_adjoint_gradient_matches_central_differences():
    """The oracle's MPFA-O adjoint (interaction-region local systems split by
    cell, its own assembly) against central differences of J through the
    independent MPFA-O assembly of the input generator, on a 4 x 3 x 3 grid
    with full anisotropic tensors, no-flow faces and two corner wells."""
    from synth.darcy import anisotropic_tensors
    from synth.fields import rotation_zyx
    rng = np.random.default_rng(31)
    dims = (4, 3, 3)
    n = int(np.prod(dims))
    K_hat = anisotropic_tensors(np.zeros(dims), rotation_zyx(20.0, 35.0, 0.0), (1.0, 1.0, 0.1))
    logk = 0.8 * rng.standard_normal(n)
    wells = [(0, 1.0), (n - 1, 0.0)]
    obs = np.array([5, 11, 17, 22, 30])
    J0, A, b = _mpfa_J(K_hat, logk, wells, obs, np.zeros(len(obs)))
    p_obs = sla.spsolve(A.tocsc(), b)[obs] + 0.05 * rng.standard_normal(len(obs))
    J, g, p = O.mpfa_objective_gradient(K_hat, logk, wells, obs, p_obs, *_mpfa_J(K_hat, logk, wells, obs, p_obs)[1:])
    h = 1e-5
    fd = np.zeros(n)
    for c in range(n):
        e = np.zeros(n)
        e[c] = h
        fd[c] = (_mpfa_J(K_hat, logk + e, wells, obs, p_obs)[0] - _mpfa_J(K_hat, logk - e, wells, obs, p_obs)[0]) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()
    assert np.abs(fd).max() > 1e-3
