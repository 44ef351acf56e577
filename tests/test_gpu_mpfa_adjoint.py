"""The MPFA-O forward model (GPU assembly) and its adjoint gradient through
the interaction regions' local systems, on the 27-point Darcy workloads.

- Assembly: the GPU's MPFA-O values and b against the input generator's
  independent assembly (1e-12 of the largest entry), wells included.
- Gradient kernel: g = -lambda^T (dA/dtheta) p + lambda^T db/dtheta against
  the oracle's (1e-10 relative) for the same lambda and p.
- dJ/d ln k of J = sum (p_obs - p)^2 over 64 observation cells (observations
  from a field perturbed by 0.1 N(0, 1)), through MsrsbMpfaSolve (MsRSB
  solves of A and A^T, each followed by two steps of iterative refinement
  with FP64 residuals): against the oracle's adjoint gradient with direct
  solves on 32^3 (1e-6 relative; solves to 1e-10), and against central
  differences of J on the 128^3 workload (sigma = 2; 1e-5 relative; solves to
  1e-8, where one Krylov solve stalls near 3e-10) along the 16 cells of
  largest sensitivity and 4 random directions."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import anisotropic_tensors, mpfa_o  # noqa: E402
from synth.fields import gaussian_random_field, rotation_zyx  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _model(dims, sigma, seed):
    rng = np.random.default_rng(seed)
    theta = gaussian_random_field(dims, 8.0, sigma, rng)
    K_hat = anisotropic_tensors(np.zeros(dims), rotation_zyx(20.0, 35.0, 0.0), (1.0, 1.0, 0.1))
    n = int(np.prod(dims))
    wells = [(0, 1.0), (n - 1, 0.0)]
    return theta.ravel(order="F"), K_hat, wells, rng


def _pattern27(dims):
    """CSR pattern of every cell's in-grid 3x3x3 neighbours, columns
    ascending (cells x fastest)."""
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


def _gpu_model(M, dims, K_hat, wells):
    n = int(np.prod(dims))
    ip, ix = _pattern27(dims)
    rowptr = torch.as_tensor(ip, device="cuda")
    colidx = torch.as_tensor(ix, device="cuda")
    Kh = torch.as_tensor(np.ascontiguousarray(np.moveaxis(K_hat, [0, 1, 2], [2, 1, 0]).reshape(n, 3, 3)), device="cuda")
    return (M.grid(dims, (8, 8, 8)), Kh, wells, rowptr, colidx), ip, ix


def _host_system(K_hat, theta, wells):
    dims = K_hat.shape[:3]
    K = np.exp(theta).reshape(dims, order="F")[..., None, None] * K_hat
    ip, ix, d, b = mpfa_o(K, {}, wells)
    return sp.csr_matrix((d, ix, ip)), b


@pytest.mark.parametrize("dims", [(12, 12, 12), (9, 7, 5)])
def test_mpfa_assembly_matches_the_generator(M, dims):
    theta, K_hat, wells, _ = _model(dims, 1.5, 5)
    model, ip, ix = _gpu_model(M, dims, K_hat, wells)
    val, b = M.msrsb.msrsb_mpfa_assemble(model[0], model[1], torch.as_tensor(theta, device="cuda"), wells,
                                         model[3], model[4])
    A, bh = _host_system(K_hat, theta, wells)
    A.sort_indices()
    assert np.array_equal(A.indptr, ip) and np.array_equal(A.indices, ix)
    assert np.abs(val.cpu().numpy() - A.data).max() <= 1e-12 * np.abs(A.data).max()
    assert np.abs(b.cpu().numpy() - bh).max() <= 1e-12 * np.abs(bh).max()


def test_mpfa_gradient_kernel_matches_oracle(M):
    dims = (10, 8, 6)
    theta, K_hat, wells, rng = _model(dims, 1.0, 6)
    n = int(np.prod(dims))
    lam, p = rng.standard_normal(n), rng.standard_normal(n)
    model, _, _ = _gpu_model(M, dims, K_hat, wells)
    g = M.msrsb.msrsb_mpfa_gradient(model[0], model[1], torch.as_tensor(theta, device="cuda"), wells,
                                    torch.as_tensor(lam, device="cuda"), torch.as_tensor(p, device="cuda")).cpu().numpy()
    K = np.exp(theta).reshape(dims, order="F")[..., None, None] * K_hat
    parts = O.mpfa_region_parts(K, dims)
    ref = -O.mpfa_lam_dA_p(parts, lam, p)
    for cell, pw in wells:
        e = np.zeros(n)
        e[cell] = 1.0
        ref -= lam[cell] * (p[cell] - pw) * O.mpfa_lam_dA_p(parts, e, e)
    assert np.linalg.norm(g - ref) <= 1e-10 * np.linalg.norm(ref)


def _objective_setup(M, dims, sigma, seed):
    theta, K_hat, wells, rng = _model(dims, sigma, seed)
    n = int(np.prod(dims))
    obs = np.sort(rng.choice(n, 64, replace=False))
    A, b = _host_system(K_hat, theta + 0.1 * rng.standard_normal(n), wells)
    import scipy.sparse.linalg as spla
    p_obs = spla.spsolve(A.tocsc(), b)[obs] if n <= 40000 else None
    return theta, K_hat, wells, obs, p_obs, rng


def _J(M, theta_t, model, obs_t, pobs_t, o, rtol):
    from paper_1912_06934_gb300.adjoint import msrsb_mpfa_solve_diff
    p = msrsb_mpfa_solve_diff(theta_t, model, o, rtol=rtol, maxit=1000, refine=2)
    return ((p[obs_t] - pobs_t) ** 2).sum()


def test_mpfa_adjoint_gradient_matches_oracle_32(M):
    dims = (32, 32, 32)
    theta, K_hat, wells, obs, p_obs, _ = _objective_setup(M, dims, 2.0, 1005)
    model, _, _ = _gpu_model(M, dims, K_hat, wells)
    o = M.opts(tol=1e-3, max_iter=100)
    th = torch.as_tensor(theta, device="cuda").requires_grad_(True)
    J = _J(M, th, model, torch.as_tensor(obs, device="cuda"), torch.as_tensor(p_obs, device="cuda"), o, 1e-10)
    (g,) = torch.autograd.grad(J, th)
    A, b = _host_system(K_hat, theta, wells)
    Jr, gr, _ = O.mpfa_objective_gradient(K_hat, theta, wells, obs, p_obs, A, b)
    assert abs(float(J.detach()) - Jr) <= 1e-8 * Jr
    assert np.linalg.norm(g.cpu().numpy() - gr) <= 1e-6 * np.linalg.norm(gr)


def test_mpfa_adjoint_gradient_matches_central_differences_128(M):
    """The 128^3 workload (2,097,152 cells, sigma = 2): the adjoint gradient
    against central differences of J, extrapolated (4 D(h/2) - D(h)) / 3 with
    h = 1e-2 (truncation error O(h^4)), each J from the GPU assembly and an
    MsRSB solve to 1e-8 with two steps of iterative refinement (true relative
    residual near 1e-11, the FP64 floor of b - A p). Checked along the unit
    vectors of the 16 cells with the largest |dJ/dtheta| and along 4 random
    N(0, 1) directions, which weigh every cell: 99.9 % of the cells have
    |dJ/dtheta| below 1e-3 of the largest, too small for a central difference
    of J in FP64 to resolve one by one."""
    dims = (128, 128, 128)
    theta, K_hat, wells, rng = _model(dims, 2.0, 1005)
    n = int(np.prod(dims))
    obs = np.sort(rng.choice(n, 64, replace=False))
    model, _, _ = _gpu_model(M, dims, K_hat, wells)
    o = M.opts(tol=1e-3, max_iter=100)
    obs_t = torch.as_tensor(obs, device="cuda")
    # observations: the solution on a field perturbed by 0.1 N(0, 1)
    th_obs = torch.as_tensor(theta + 0.1 * rng.standard_normal(n), device="cuda")
    from paper_1912_06934_gb300.adjoint import msrsb_mpfa_solve_diff
    with torch.no_grad():
        pobs_t = msrsb_mpfa_solve_diff(th_obs, model, o, rtol=1e-8, maxit=500, refine=2)[obs_t].clone()
    th = torch.as_tensor(theta, device="cuda").requires_grad_(True)
    J = _J(M, th, model, obs_t, pobs_t, o, 1e-8)
    (g,) = torch.autograd.grad(J, th)
    th = th.detach()

    def D(v, h):
        with torch.no_grad():
            return (float(_J(M, th + h * v, model, obs_t, pobs_t, o, 1e-8)) -
                    float(_J(M, th - h * v, model, obs_t, pobs_t, o, 1e-8))) / (2 * h)

    def richardson(v, h=1e-2):
        return (4 * D(v, h / 2) - D(v, h)) / 3

    cells = torch.argsort(g.abs(), descending=True)[:16]
    fd = []
    for c in cells.tolist():
        e = torch.zeros_like(th)
        e[c] = 1.0
        fd.append(richardson(e))
    fd = np.array(fd)
    assert np.linalg.norm(g[cells].cpu().numpy() - fd) <= 1e-5 * np.linalg.norm(fd)
    for _ in range(4):
        v = torch.as_tensor(rng.standard_normal(n), device="cuda")
        gv = float(torch.dot(g, v))
        fdv = richardson(v)
        assert abs(gv - fdv) <= 1e-5 * abs(fdv)
