"""Several right-hand sides in lockstep (msrsb_solve_multi): every right-hand
side performs exactly the operations of its own msrsb_solve, so iterations
and solutions must equal those of the individual solves bit for bit; mixed
and FP64 forms, a batch of 5 and a split batch of 11 (8 + 3); and the
one-after-another fallback for a configuration the multi-vector kernels do
not serve (PCG with block Gauss-Seidel)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth.darcy import darcy_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _rhs(c, k, seed):
    import scipy.sparse as sp
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    xi = np.random.default_rng(seed).standard_normal((k, A.shape[0]))
    return np.ascontiguousarray((A @ xi.T).T)


@pytest.mark.parametrize("prec,k", [(1, 5), (0, 5), (1, 11)])
def test_multi_equals_individual_solves(M, prec, k):
    c = darcy_3d_case(dims=(40, 24, 20), H=8, seed=5)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    h = M.msrsb_setup(A, g, M.opts(prec=prec, tol=1e-3, max_iter=100))
    B = torch.as_tensor(_rhs(c, k, 11 + k), device="cuda")
    out = h.solve_multi(B, rtol=1e-8, maxit=300)
    for r in range(k):
        one = h.solve(B[r].clone(), rtol=1e-8, maxit=300)
        assert out["iters"][r] == one["iters"], (r, out["iters"][r], one["iters"])
        assert torch.equal(out["x"][r], one["x"]), r
        assert out["relres"][r] == one["relres"]
        assert out["relres"][r] <= 1e-8
    h.destroy()


def test_multi_falls_back_to_individual_solves(M):
    from synth.elastic import elastic_3d_case
    B_ = M.msrsb
    c = elastic_3d_case(ne=8, H=4)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=3)
    g = M.grid(c["dims"], c["H"], centering=1, ncomp=3)
    h = M.msrsb_setup(A, g, M.opts(krylov=B_.MSRSB_PCG, smoother=B_.MSRSB_SMOOTH_GS, pre=1, post=1))
    N = len(c["b"])
    B = torch.as_tensor(np.random.default_rng(3).standard_normal((3, N)), device="cuda")
    out = h.solve_multi(B, rtol=1e-8, maxit=300)
    for r in range(3):
        one = h.solve(B[r].clone(), rtol=1e-8, maxit=300)
        assert out["iters"][r] == one["iters"]
        assert torch.equal(out["x"][r], one["x"])
    h.destroy()
