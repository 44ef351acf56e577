"""Parity at the configurations' full sizes, in the benchmark's launch
configuration.

- 3D Darcy 64^3 (262,144 cells, the benchmark's workload): the oracle's full
  FP64 set-up (100 Alg. 1 passes, tol 1e-3) and right-preconditioned GMRES
  solve to 1e-8 are compared with the GPU's FP64 form (P within 1e-11) and
  mixed form (P within 1e-5); both must reach relative residual 1e-8,
  recomputed here in FP64, within +-1 iteration of the oracle.
- 3D elasticity 48^3 Q1 elements (352,947 dofs): one GPU smoothing pass of
  every SDC component equals the oracle's pass applied to the GPU's previous
  iterate; the PCG solve (block Gauss-Seidel pre/post) reaches 1e-8 within
  +-1 of the oracle's iteration count in both forms.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import darcy_3d_case  # noqa: E402
from synth.elastic import elastic_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu

BASIS = dict(tol=1e-3, n_it=10, max_iter=100)


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


def _on_pattern(Pm, pat):
    Pm = Pm.tocsr()
    Pm.sort_indices()
    return np.asarray(Pm[np.repeat(np.arange(Pm.shape[0]), np.diff(pat.indptr)), pat.indices]).ravel()


@pytest.fixture(scope="module")
def darcy64():
    c = darcy_3d_case(n=64)
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    A.sort_indices()
    ref = O.setup_scalar(A, c["dims"], c["H"], **BASIS)
    x, its, rr, _ = O.gmres_right(A, c["b"], ref["tl"].apply, rtol=1e-8, maxit=300)
    return c, A, ref, its


@pytest.mark.parametrize("prec", [0, 1])
def test_darcy64_setup_and_gmres_match_oracle(M, darcy64, prec):
    c, A, ref, its_ref = darcy64
    Ad = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    h = M.msrsb_setup(Ad, g, M.opts(prec=prec, **BASIS))
    info = h.info()
    # FP32 passes may meet the tolerance at a neighbouring check
    assert abs(info["basis_iters"] - ref["iters"]) <= (0 if prec == 0 else BASIS["n_it"])
    p_ids, p_val, _ = h.get_setup()
    nc = ref["part"]["nc"]
    diff = np.abs(_gpu_P(p_ids, p_val[0], nc) - ref["P"]).max()
    assert diff <= (1e-11 if prec == 0 else 1e-5)
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=300)
    x = r["x"].cpu().numpy()
    relres = np.linalg.norm(c["b"] - A @ x) / np.linalg.norm(c["b"])
    assert relres <= 1e-8
    assert abs(r["iters"] - its_ref) <= 1
    h.destroy()


@pytest.fixture(scope="module")
def elastic48():
    return elastic_3d_case(ne=48, H=6)


def _elastic_setup(M, c, prec, **kw):
    from paper_1912_06934_gb300 import msrsb as B
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=3)
    g = M.grid(c["dims"], c["H"], centering=1, ncomp=3)
    o = M.opts(prec=prec, smoother=B.MSRSB_SMOOTH_GS, pre=1, post=1, krylov=B.MSRSB_PCG, **kw)
    return A, M.msrsb_setup(A, g, o)


def test_elastic48_one_pass_per_component(M, elastic48):
    c = elastic48
    k = 4
    _, hk = _elastic_setup(M, c, 0, tol=0.0, max_iter=k)
    _, hk1 = _elastic_setup(M, c, 0, tol=0.0, max_iter=k + 1)
    p_ids, Pk, _ = hk.get_setup()
    _, Pk1, _ = hk1.get_setup()
    part = O.partition(c["dims"], c["H"], 1)
    pat, nc = part["pat"], part["nc"]
    comps = O.sdc_blocks(c["indptr"], c["indices"], c["data"])
    for l in range(3):
        Ah = O.mmatrix_filter(comps[l])
        vals_k = _on_pattern(_gpu_P(p_ids, Pk[l], nc), pat)
        nxt, _ = O.smoothing_pass(Ah, pat, vals_k, O.inverse_diagonal(Ah), 2.0 / 3.0)
        got = _on_pattern(_gpu_P(p_ids, Pk1[l], nc), pat)
        assert np.abs(got - nxt).max() <= 1e-13
        Pn = O.as_matrix(got, pat)
        assert np.abs(np.asarray(Pn.sum(axis=1)).ravel() - 1).max() <= 1e-14
    hk.destroy()
    hk1.destroy()


def test_elastic48_pcg(M, elastic48):
    c = elastic48
    A = O.bsr_to_csr(c["indptr"], c["indices"], c["data"])
    b = c["b"]
    ref = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], **BASIS)
    _, its_ref, rr_ref, _ = O.pcg(A, b, ref["tl"].apply, rtol=1e-8, maxit=500)
    assert rr_ref <= 1e-8
    for prec in (0, 1):
        _, h = _elastic_setup(M, c, prec, **BASIS)
        r = h.solve(torch.as_tensor(b, device="cuda"), rtol=1e-8, maxit=500)
        x = r["x"].cpu().numpy()
        assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-8
        assert abs(r["iters"] - its_ref) <= 1, (prec, r["iters"], its_ref)
        h.destroy()
