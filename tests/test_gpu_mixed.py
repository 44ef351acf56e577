"""The mixed-precision form (FP32 basis, P, smoother and inner residuals;
FP64 Krylov vectors, coarse operator and coarse solve) against the FP64
oracle, each result with its stated error bound.

Bounds. FP32 P is within 1e-5 max-abs of the oracle's FP64 P (the FP32
tolerance on P). A_c = P^T A P and the two-stage apply are linear in P on each
side, so to first order their relative error is at most twice P's relative
error, plus FP32 rounding of the smoother (unit roundoff 6e-8, amplified by
the sweep's ~27-term sums): 2e-5 relative is the stated bound for A_c
(Frobenius) and for one application of the preconditioner (2-norm). The solve
is judged as in the FP64 form: true relative residual <= 1e-8 (recomputed
here) and the oracle's iteration count within +-1.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import darcy_3d_case  # noqa: E402
from synth.elastic import elastic_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu

P_TOL32 = 1e-5
AC_TOL32 = 2e-5
APPLY_TOL32 = 2e-5


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _gpu_P(p_ids, p_val, nc):
    ids = p_ids.cpu().numpy()
    vals = p_val.cpu().numpy().astype(np.float64)
    rows, slots = np.nonzero(ids >= 0)
    return sp.csr_matrix((vals[rows, slots], (rows, ids[rows, slots])), shape=(ids.shape[0], nc))


def _block_gpu_P(p_ids, p_val, nc):
    return O.block_prolongation([_gpu_P(p_ids, p_val[l], nc) for l in range(3)])


@pytest.mark.parametrize("case", ["scalar24", "elastic12"])
def test_mixed_results_match_oracle(M, case):
    B = M.msrsb
    basis = dict(tol=1e-3, n_it=10, max_iter=100)
    if case == "scalar24":
        c = darcy_3d_case(n=24)
        A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
        g = M.grid(c["dims"], c["H"])
        o = M.opts(prec=B.MSRSB_F32, **basis)
        Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
        ref = O.setup_scalar(Ah, c["dims"], c["H"], **basis)
        nc = ref["part"]["nc"]
        solve = O.gmres_right
    else:
        c = elastic_3d_case(ne=12, H=6)
        A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=3)
        g = M.grid(c["dims"], c["H"], centering=1, ncomp=3)
        o = M.opts(prec=B.MSRSB_F32, smoother=B.MSRSB_SMOOTH_GS, pre=1, post=1, krylov=B.MSRSB_PCG, **basis)
        ref = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], **basis)
        Ah = ref["A"]
        nc = ref["part"]["nc"]
        solve = O.pcg
    h = M.msrsb_setup(A, g, o)
    p_ids, p_val, Ac = h.get_setup()
    if case == "scalar24":
        Pg, Po = _gpu_P(p_ids, p_val[0], nc), ref["P"]
    else:
        Pg, Po = _block_gpu_P(p_ids, p_val, nc), ref["P"]
    assert abs(Pg - Po).max() <= P_TOL32
    Aco = ref["tl"].Ac.toarray()
    assert np.linalg.norm(Ac.cpu().numpy() - Aco) <= AC_TOL32 * np.linalg.norm(Aco)
    v = np.random.default_rng(21).standard_normal(Ah.shape[0])
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = ref["tl"].apply(v)
    assert np.linalg.norm(z - zr) <= APPLY_TOL32 * np.linalg.norm(zr)
    _, its_ref, _, _ = solve(Ah, c["b"], ref["tl"].apply, rtol=1e-8, maxit=500)
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=500)
    x = r["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"])
    assert abs(r["iters"] - its_ref) <= 1, (r["iters"], its_ref)
    h.destroy()
