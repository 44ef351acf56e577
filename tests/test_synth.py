"""Pins for the shared input generators (not part of the method)."""
import numpy as np
import scipy.sparse as sp

from synth.darcy import mpfa_o, tpfa, darcy_2d_case
from synth.elastic import q1_elasticity
from synth.fields import rotation_zyx, gaussian_random_field


def _dense(t):
    return sp.csr_matrix((t[2], t[1], t[0])).toarray()


def test_mpfa_equals_tpfa_for_diagonal_K():
    # MPFA-O on K-orthogonal Cartesian grids reduces to TPFA (Sec. 3.1).
    rng = np.random.default_rng(3)
    for dims in [(5, 4), (4, 3, 5)]:
        d = len(dims)
        K = np.zeros(dims + (d, d))
        for a in range(d):
            K[..., a, a] = np.exp(rng.standard_normal(dims))
        bc = {(0, 0): ("D", 1.0), (0, 1): ("D", 0.0)}
        A1, A2 = mpfa_o(K, bc), tpfa(K, bc)
        assert np.abs(_dense(A1) - _dense(A2)).max() < 1e-12
        assert np.abs(A1[3] - A2[3]).max() < 1e-12


def test_mpfa_reproduces_linear_fields():
    # consistency of the O-method: a linear pressure field has zero flux
    # divergence in cells away from the boundary, for any constant full tensor
    for dims in [(6, 5), (5, 4, 6)]:
        d = len(dims)
        R = rotation_zyx(20, 35, 0)[:d, :d] if d == 3 else np.array([[np.cos(.5), -np.sin(.5)], [np.sin(.5), np.cos(.5)]])
        K0 = R @ np.diag([1.0, 0.3, 0.1][:d]) @ R.T
        K = np.broadcast_to(K0, dims + (d, d)).copy()
        ip, ix, dv, _ = mpfa_o(K, {})
        A = sp.csr_matrix((dv, ix, ip))
        X = np.indices(dims).reshape(d, -1, order="F") + 0.5
        r = A @ (np.array([0.3, -0.7, 0.2][:d]) @ X)
        inner = np.ones(X.shape[1], bool)
        for a in range(d):
            inner &= (X[a] > 1) & (X[a] < dims[a] - 1)
        assert np.abs(r[inner]).max() < 1e-12
        assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-12


def test_darcy_2d_has_positive_offdiagonals():
    c = darcy_2d_case()
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    off = A - sp.diags(A.diagonal())
    assert (off.data > 0).sum() > 0.1 * A.nnz  # not an M-matrix
    assert A.nnz == (3 * 64 - 2) ** 2


def test_q1_rigid_modes_and_spd():
    e = q1_elasticity(np.ones((3, 3, 3)), 0.25 * np.ones((3, 3, 3)), fixed_bottom=False, top_traction=None)
    A = sp.bsr_matrix((e["data"], e["indices"], e["indptr"])).toarray()
    X = np.indices(e["node_dims"]).reshape(3, -1, order="F").T.astype(float)
    modes = [np.tile([1, 0, 0], len(X)), np.tile([0, 1, 0], len(X)), np.tile([0, 0, 1], len(X)),
             np.stack([-X[:, 1], X[:, 0], 0 * X[:, 0]], 1).ravel(),
             np.stack([0 * X[:, 0], -X[:, 2], X[:, 1]], 1).ravel(),
             np.stack([X[:, 2], 0 * X[:, 0], -X[:, 0]], 1).ravel()]
    for v in modes:
        assert np.abs(A @ v).max() < 1e-12
    w = np.linalg.eigvalsh(A)
    assert np.sum(np.abs(w) < 1e-10) == 6 and w[6] > 1e-3
    assert np.abs(A - A.T).max() == 0.0


def test_q1_fixed_bottom_is_spd():
    rng = np.random.default_rng(0)
    e = q1_elasticity(np.exp(rng.standard_normal((3, 2, 2))), rng.uniform(0.2, 0.35, (3, 2, 2)))
    A = sp.bsr_matrix((e["data"], e["indices"], e["indptr"])).toarray()
    assert np.abs(A - A.T).max() == 0.0
    assert np.linalg.eigvalsh(A).min() > 0
    # total applied load equals traction x top area
    assert abs(e["b"].reshape(-1, 3)[:, 2].sum() + 3 * 2) < 1e-12


def test_grf_statistics():
    f = gaussian_random_field((64, 64), 8.0, 3.0, np.random.default_rng(1))
    assert abs(f.std() - 3.0) < 1e-12 and abs(f.mean()) < 1e-12
    # strongly correlated at one cell, nearly uncorrelated at 3 correlation lengths
    c1 = np.corrcoef(f[:-1].ravel(), f[1:].ravel())[0, 1]
    c24 = np.corrcoef(f[:-24].ravel(), f[24:].ravel())[0, 1]
    assert c1 > 0.9 and abs(c24) < 0.3


# ---------------- MPFA-O on rough quadrilateral grids (Sec. 3.1, 3.2) ----------------

def test_quad_mpfa_equals_the_cartesian_generator_on_a_unit_grid():
    """Two independent MPFA-O assemblies agree where both apply: the general
    quadrilateral one on an unperturbed grid of unit cells and the Cartesian
    one, full rotated tensors, Dirichlet on x = min / max, no flow elsewhere."""
    from synth.darcy import mpfa_o, mpfa_o_quads, anisotropic_tensors
    from synth.fields import rotation_2d
    rng = np.random.default_rng(3)
    n = 7
    K = anisotropic_tensors(rng.standard_normal((n, n)), rotation_2d(30.0), (1.0, 0.1))
    bc = {(0, 0): ("D", 1.0), (0, 1): ("D", 0.0)}
    a = mpfa_o(K, bc)
    X, Y = np.meshgrid(np.arange(n + 1) * 1.0, np.arange(n + 1) * 1.0, indexing="ij")
    q = mpfa_o_quads(X, Y, K, bc)
    A1 = sp.csr_matrix((a[2], a[1], a[0])).toarray()
    A2 = sp.csr_matrix((q[2], q[1], q[0])).toarray()
    assert np.abs(A1 - A2).max() <= 1e-13 * np.abs(A1).max()
    assert np.abs(a[3] - q[3]).max() <= 1e-13


def test_quad_mpfa_is_exact_for_linear_pressure_on_a_perturbed_grid():
    """MPFA-O reproduces linear pressure fields on rough grids with a constant
    full tensor (its defining consistency), with Dirichlet data from the field."""
    from synth.darcy import mpfa_o_quads, perturbed_grid
    rng = np.random.default_rng(4)
    nx, ny = 12, 9
    X, Y = perturbed_grid(nx, ny, 3.0, 5.0, 0.4, rng)
    assert np.abs(X[1:-1, 1:-1] - np.arange(1, nx)[:, None] * 0.25).max() > 1e-3  # really perturbed
    K = np.broadcast_to(np.array([[2.0, 0.7], [0.7, 1.0]]), (nx, ny, 2, 2)).copy()

    def f(x, y):
        return 0.3 + 1.7 * x - 0.9 * y

    bc = {(ax, sd): ("D", f) for ax in (0, 1) for sd in (0, 1)}
    ip, ix, d, b = mpfa_o_quads(X, Y, K, bc)
    A = sp.csr_matrix((d, ix, ip))
    xc = 0.25 * (X[:-1, :-1] + X[1:, :-1] + X[1:, 1:] + X[:-1, 1:])
    yc = 0.25 * (Y[:-1, :-1] + Y[1:, :-1] + Y[1:, 1:] + Y[:-1, 1:])
    p = f(xc, yc).T.ravel()  # cells flat i + nx*j
    assert np.abs(A @ p - b).max() <= 1e-12 * np.abs(b).max()


def test_paper_mpfa_case_is_not_an_m_matrix_and_conserves():
    """The Sec. 3.2 case: 100 x 100 rough cells, tensor [[100, 25], [25, 100]];
    interior rows sum to zero (no flow, no Dirichlet half-edge) and a large
    share of off-diagonals is positive, so A is not an M-matrix."""
    from synth.darcy import darcy_2d_perturbed_case
    c = darcy_2d_perturbed_case()
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    assert A.shape == (10000, 10000)
    n = 100
    i = np.arange(n * n) % n
    interior = (i > 0) & (i < n - 1)
    rs = np.asarray(A.sum(axis=1)).ravel()
    assert np.abs(rs[interior]).max() <= 1e-12 * np.abs(A.diagonal()).max()
    off = A - sp.diags(A.diagonal())
    assert (off.data > 0).mean() > 0.2
