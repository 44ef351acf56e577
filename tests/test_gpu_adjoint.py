"""Adjoint support: A^T's values in A's pattern, the pattern outer product,
the differentiable MsRSB solve (MsrsbSolve) and the gradient of a pressure
misfit with respect to log-permeability through the two-point flux model.

Checks: A^T values and lambda x^T bit for bit against scipy/numpy; dJ/db and
dJ/dA of J = w.x against direct solves (1e-8 relative; solves to 1e-11 on a
sigma = 1 field); dJ/d log k on a 32^3 field (sigma = 2, 64 observation cells,
observations from a perturbed field) against the oracle's adjoint (1e-6
relative) and against central differences on 32 random cells (1e-5 relative)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import _grid_flat, darcy_3d_case  # noqa: E402
from synth.elastic import elastic_3d_case  # noqa: E402
from synth.fields import gaussian_random_field  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _entries(indptr, indices):
    rows = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    return rows, np.asarray(indices)


def test_transpose_values_and_pattern_outer(M):
    c = darcy_3d_case(n=12)  # MPFA-O: symmetric pattern, non-symmetric values
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    rows, cols = _entries(c["indptr"], c["indices"])
    vt = M.msrsb.msrsb_transpose_values(A).cpu().numpy()
    assert np.array_equal(vt, np.asarray(Ah.T.tocsr()[rows, cols]).ravel())
    rng = np.random.default_rng(1)
    lam, x = rng.standard_normal(Ah.shape[0]), rng.standard_normal(Ah.shape[0])
    g = M.msrsb.msrsb_pattern_outer(A, -1.0, torch.as_tensor(lam, device="cuda"),
                                    torch.as_tensor(x, device="cuda")).cpu().numpy()
    assert np.array_equal(g, -1.0 * lam[rows] * x[cols])
    # 3x3 blocks: block (i, j) of A^T is block (j, i) of A, transposed
    e = elastic_3d_case(ne=3, H=2)
    Ab = M.Mat.from_host(e["indptr"], e["indices"], e["data"], bdim=3)
    vb = M.msrsb.msrsb_transpose_values(Ab).cpu().numpy().reshape(-1, 3, 3)
    Bs = sp.bsr_matrix((e["data"], e["indices"], e["indptr"]))
    Bt = Bs.T.tobsr(blocksize=(3, 3))
    Bt.sort_indices()
    br, bc = _entries(e["indptr"], e["indices"])
    D = Bt.toarray()
    for q in range(0, len(br), 97):
        assert np.array_equal(vb[q], D[3 * br[q]:3 * br[q] + 3, 3 * bc[q]:3 * bc[q] + 3])
    # a pattern without a mirror entry is refused
    ip, ix = np.array([0, 2, 3], dtype=np.int32), np.array([0, 1, 1], dtype=np.int32)
    Ans = M.Mat.from_host(ip, ix, np.array([2.0, -1.0, 2.0]))
    with pytest.raises(M.MsrsbError) as ei:
        M.msrsb.msrsb_transpose_values(Ans)
    assert ei.value.status == M.msrsb.MSRSB_ESHAPE


def test_msrsb_solve_gradients_nonsymmetric(M):
    from paper_1912_06934_gb300.adjoint import msrsb_solve_diff
    c = darcy_3d_case(n=16, sigma=1.0)  # sigma 1: relres 1e-11 is reachable in FP64
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    rows, cols = _entries(c["indptr"], c["indices"])
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    vals = A.val.clone().requires_grad_(True)
    b = torch.as_tensor(c["b"], device="cuda").requires_grad_(True)
    o = M.opts(tol=1e-3, max_iter=100)
    x = msrsb_solve_diff(vals, b, (A.rowptr, A.colidx, 1, g), o, rtol=1e-11, maxit=500)
    w = torch.as_tensor(np.random.default_rng(2).standard_normal(Ah.shape[0]), device="cuda")
    (w * x).sum().backward()
    x_ref = spla.spsolve(Ah.tocsc(), c["b"])
    lam_ref = spla.spsolve(Ah.T.tocsc(), w.cpu().numpy())
    assert np.linalg.norm(x.detach().cpu().numpy() - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert np.linalg.norm(b.grad.cpu().numpy() - lam_ref) <= 1e-8 * np.linalg.norm(lam_ref)
    gv = -lam_ref[rows] * x_ref[cols]
    assert np.linalg.norm(vals.grad.cpu().numpy() - gv) <= 1e-8 * np.linalg.norm(gv)


def _c5_like(n, seed=1005):
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    logk = _grid_flat(gaussian_random_field(dims, 8.0, 2.0, rng), dims)
    ncell = n ** 3
    obs = np.sort(rng.choice(ncell, size=64, replace=False))
    pert = logk + 0.1 * rng.standard_normal(ncell)
    _, _, p_pert = O.tpfa_objective_gradient(dims, pert, obs, np.zeros(64))
    return dims, logk, obs, p_pert[obs]


def test_log_perm_gradient_against_oracle_and_differences(M):
    from paper_1912_06934_gb300.adjoint import msrsb_solve_diff, tpfa_darcy, tpfa_pattern
    dims, logk, obs, p_obs = _c5_like(32)
    pat = tpfa_pattern(dims)
    g = M.grid(dims, (8, 8, 8))
    o = M.opts(tol=1e-3, max_iter=100)
    obs_t = torch.as_tensor(obs, device="cuda")
    pobs_t = torch.as_tensor(p_obs, device="cuda")

    def objective(theta, grad):
        th = torch.as_tensor(theta, device="cuda").requires_grad_(grad)
        vals, b = tpfa_darcy(th, pat)
        x = msrsb_solve_diff(vals, b, (pat["rowptr"], pat["colidx"], 1, g), o, rtol=1e-13, maxit=1000)
        J = ((x[obs_t] - pobs_t) ** 2).sum()
        if grad:
            J.backward()
            return float(J.detach()), th.grad.cpu().numpy()
        return float(J.detach()), None

    J, grad = objective(logk, True)
    J_ref, g_ref, _ = O.tpfa_objective_gradient(dims, logk, obs, p_obs)
    assert abs(J - J_ref) <= 1e-9 * abs(J_ref)
    assert np.linalg.norm(grad - g_ref) <= 1e-6 * np.linalg.norm(g_ref)
    rng = np.random.default_rng(6)
    cells = rng.choice(len(logk), size=32, replace=False)
    eps = 1e-4
    scale = np.abs(g_ref).max()
    for cidx in cells:
        e = np.zeros_like(logk)
        e[cidx] = eps
        fd = (objective(logk + e, False)[0] - objective(logk - e, False)[0]) / (2 * eps)
        assert abs(grad[cidx] - fd) <= 1e-5 * max(abs(fd), 1e-3 * scale)
