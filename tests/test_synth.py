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
