"""Second-stage variants of Sec. 3.2 and Sec. 4 against the oracle: the
l1-Jacobi smoother (pre and post sweeps), the smoothing-only baseline (no
multiscale stage), and the stand-alone Richardson iteration.

Tolerances as in test_gpu_parity: one application of the preconditioner within
1e-10 relative (FP64 form); Krylov/Richardson solves to relative residual 1e-8
(recomputed here) with iteration counts within +-1 of the oracle's."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import darcy_2d_case, darcy_3d_case  # noqa: E402
from synth.elastic import elastic_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _elastic(M, c, **kw):
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=3)
    g = M.grid(c["dims"], c["H"], centering=1, ncomp=3)
    return M.msrsb_setup(A, g, M.opts(**kw))


@pytest.mark.parametrize("coarse", [1, 0])
def test_l1_jacobi_apply_matches_oracle_elastic(M, coarse):
    B = M.msrsb
    c = elastic_3d_case(ne=8, H=4)
    h = _elastic(M, c, smoother=B.MSRSB_SMOOTH_L1JAC, pre=2, post=2, krylov=B.MSRSB_PCG, tol=0.0, max_iter=20,
                 no_coarse=1 - coarse)
    ref = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], tol=0.0, max_iter=20,
                          smoother="l1jac", sweeps=2, coarse=bool(coarse))
    v = np.random.default_rng(5).standard_normal(ref["A"].shape[0])
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = ref["tl"].apply(v)
    assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr)
    h.destroy()


def test_l1_jacobi_apply_matches_oracle_scalar(M):
    B = M.msrsb
    c = darcy_3d_case(n=16)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    h = M.msrsb_setup(A, M.grid(c["dims"], c["H"]),
                      M.opts(smoother=B.MSRSB_SMOOTH_L1JAC, pre=1, post=3, tol=0.0, max_iter=20))
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    ref = O.setup_scalar(Ah, c["dims"], c["H"], tol=0.0, max_iter=20, smoother=None)
    tl = O.TwoLevel(Ah, ref["P"], pre=O.L1Jacobi(Ah, 1), post=O.L1Jacobi(Ah, 3))
    v = np.random.default_rng(6).standard_normal(Ah.shape[0])
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = tl.apply(v)
    assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr)
    h.destroy()


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_l1_jacobi_elastic(M, prec):
    B = M.msrsb
    c = elastic_3d_case(ne=12, H=6)
    h = _elastic(M, c, smoother=B.MSRSB_SMOOTH_L1JAC, pre=2, post=2, krylov=B.MSRSB_PCG, tol=1e-3, max_iter=100,
                 prec=prec)
    ref = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], tol=1e-3, max_iter=100,
                          smoother="l1jac", sweeps=2)
    _, its_ref, _, _ = O.pcg(ref["A"], c["b"], ref["tl"].apply, rtol=1e-8, maxit=500)
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=500)
    x = r["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - ref["A"] @ x) <= 1e-8 * np.linalg.norm(c["b"])
    # both forms within +-1 of the FP64 oracle's count
    assert abs(r["iters"] - its_ref) <= 1
    h.destroy()


def test_richardson_matches_oracle_and_beats_smoothing_only(M):
    B = M.msrsb
    c = darcy_2d_case()
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    ref = O.setup_scalar(Ah, c["dims"], c["H"], tol=1e-3, max_iter=100)
    _, its_ref, _, _ = O.richardson(Ah, c["b"], ref["tl"].apply, rtol=1e-8, maxit=300)
    h = M.msrsb_setup(A, g, M.opts(krylov=B.MSRSB_RICHARDSON, tol=1e-3, max_iter=100))
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=300)
    x = r["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"])
    assert abs(r["iters"] - its_ref) <= 1
    h.destroy()
    # smoothing only (ILU(0) alone): no convergence within 150 iterations
    h = M.msrsb_setup(A, g, M.opts(krylov=B.MSRSB_RICHARDSON, tol=1e-3, max_iter=100, no_coarse=1))
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=150, raise_on_noconv=False)
    assert r["iters"] == 150 and r["relres"] > 1e-8
    h.destroy()


def test_bad_smoother_options_are_rejected(M):
    c = darcy_2d_case(n=16, H=4)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    for kw in (dict(smoother=7), dict(pre=-1), dict(post=65), dict(no_coarse=2)):
        with pytest.raises(M.MsrsbError) as ei:
            M.msrsb_setup(A, g, M.opts(**kw))
        assert ei.value.status == M.msrsb.MSRSB_EINVAL


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("prec", [0, 1])
def test_fv_restriction_matches_oracle(M, case, prec):
    """The Petrov-Galerkin (finite-volume) restriction of Alg. 2: A_c = R A P
    with R the primal-block indicator, against the oracle: A_c within 1e-12 of
    its largest entry and one apply within 1e-10 (FP64 form; 2e-5 mixed, the
    bound of the mixed-form tests), GMRES to 1e-8 within +-1 iteration."""
    B = M.msrsb
    c = darcy_2d_case(n=64, H=8) if case == "2d" else darcy_3d_case(n=24)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    basis = dict(tol=1e-3, n_it=10, max_iter=100)
    h = M.msrsb_setup(A, g, M.opts(restriction=B.MSRSB_RESTRICT_FV, prec=prec, **basis))
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    ref = O.setup_scalar(Ah, c["dims"], c["H"], restriction="fv", **basis)
    _, _, Ac = h.get_setup()
    Acr = ref["tl"].Ac.toarray()
    assert np.abs(Ac.cpu().numpy() - Acr).max() <= (1e-12 if prec == 0 else 2e-5) * np.abs(Acr).max()
    v = np.random.default_rng(9).standard_normal(Ah.shape[0])
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = ref["tl"].apply(v)
    assert np.linalg.norm(z - zr) <= (1e-10 if prec == 0 else 2e-5) * np.linalg.norm(zr)
    _, its_ref, _, _ = O.gmres_right(Ah, c["b"], ref["tl"].apply, rtol=1e-8, maxit=300)
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=300)
    x = r["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"])
    assert abs(r["iters"] - its_ref) <= 1
    h.destroy()


def test_fv_restriction_with_pcg_is_rejected(M):
    B = M.msrsb
    c = elastic_3d_case(ne=4, H=2)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=3)
    g = M.grid(c["dims"], c["H"], centering=1, ncomp=3)
    with pytest.raises(M.MsrsbError) as ei:
        M.msrsb_setup(A, g, M.opts(smoother=B.MSRSB_SMOOTH_GS, pre=1, post=1, krylov=B.MSRSB_PCG,
                                   restriction=B.MSRSB_RESTRICT_FV))
    assert ei.value.status == B.MSRSB_EINVAL


@pytest.mark.parametrize("ne,H", [(8, 4), (12, 6)])
def test_ic0_apply_matches_oracle_elastic(M, ne, H):
    """IC(0) pre/post (Sec. 4.1, 4.3): the GPU's 3x3-block incomplete
    factorisation in the node colour order against the oracle's pointwise
    ILU(0) of the SPD operator in the same order (IC(0)); one application of
    the two-stage operator within 1e-10 relative."""
    B = M.msrsb
    c = elastic_3d_case(ne=ne, H=H)
    h = _elastic(M, c, smoother=B.MSRSB_SMOOTH_IC0, pre=1, post=1, krylov=B.MSRSB_PCG, tol=0.0, max_iter=20)
    ref = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], tol=0.0, max_iter=20,
                          smoother="ic0")
    v = np.random.default_rng(12).standard_normal(ref["A"].shape[0])
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = ref["tl"].apply(v)
    assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr)
    h.destroy()


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_ic0_elastic(M, prec):
    """PCG with IC(0) pre/post to 1e-8, within +-1 of the oracle's count."""
    B = M.msrsb
    c = elastic_3d_case(ne=16, H=4)
    basis = dict(tol=1e-3, n_it=10, max_iter=100)
    h = _elastic(M, c, smoother=B.MSRSB_SMOOTH_IC0, pre=1, post=1, krylov=B.MSRSB_PCG, prec=prec, **basis)
    ref = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], smoother="ic0", **basis)
    _, its_ref, _, _ = O.pcg(ref["A"], c["b"], ref["tl"].apply, rtol=1e-8, maxit=500)
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=500)
    x = r["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - ref["A"] @ x) <= 1e-8 * np.linalg.norm(c["b"])
    assert abs(r["iters"] - its_ref) <= 1, (r["iters"], its_ref)
    h.destroy()


def test_ic0_on_a_scalar_operator_is_ilu0(M):
    """For a scalar operator IC0 is ILU(0) (identical for a symmetric A):
    the same code path, so the applications agree bit for bit."""
    B = M.msrsb
    c = darcy_3d_case(n=16)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    v = torch.as_tensor(np.random.default_rng(13).standard_normal(A.nrows), device="cuda")
    z = []
    for sm in (B.MSRSB_SMOOTH_ILU0, B.MSRSB_SMOOTH_IC0):
        h = M.msrsb_setup(A, g, M.opts(smoother=sm, tol=0.0, max_iter=10))
        z.append(h.apply(v).cpu().numpy())
        h.destroy()
    assert np.array_equal(z[0], z[1])


@pytest.mark.parametrize("case", ["3d_ragged", "2d"])
@pytest.mark.parametrize("ordering", [0, 1])
def test_ilu0_orderings_match_oracle(M, case, ordering):
    """The ILU(0) smoother in both elimination orders against the oracle's
    factorisation in the same order: line blocks (default) and parity colours;
    one application within 1e-10 relative (FP64 form). The ragged 3D grid has
    odd y and z extents (partial line blocks) and x-lines longer than 32."""
    B = M.msrsb
    c = darcy_3d_case(dims=(40, 7, 5), H=4) if case == "3d_ragged" else darcy_2d_case(n=40, H=8)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    h = M.msrsb_setup(A, g, M.opts(tol=0.0, max_iter=20, ordering=ordering))
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    ref = O.setup_scalar(Ah, c["dims"], c["H"], tol=0.0, max_iter=20,
                         order="lines" if ordering == B.MSRSB_ORDER_LINES else "colour")
    v = np.random.default_rng(14).standard_normal(Ah.shape[0])
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = ref["tl"].apply(v)
    assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr)
    h.destroy()


@pytest.mark.parametrize("ordering", [0, 1])
def test_ordered_smoothers_reject_wide_patterns(M, ordering):
    """A coupling two points apart along x (outside the 3^d neighbourhood)
    would couple points of one colour: set-up refuses it with MSRSB_EINVAL for
    the ILU(0) smoother in either order, and l1-Jacobi (pointwise) accepts it."""
    B = M.msrsb
    c = darcy_2d_case(n=24, H=8)
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    n = Ah.shape[0]
    i = np.arange(n)
    far = (i % 24) < 22
    W = sp.csr_matrix((np.full(far.sum(), -1e-3), (i[far], i[far] + 2)), shape=(n, n))
    Aw = sp.csr_matrix(Ah + W + W.T + sp.diags(np.full(n, 2e-3)))
    Aw.sort_indices()
    A = M.Mat.from_host(Aw.indptr, Aw.indices, Aw.data)
    g = M.grid(c["dims"], c["H"])
    with pytest.raises(M.MsrsbError) as e:
        M.msrsb_setup(A, g, M.opts(ordering=ordering))
    assert e.value.status == B.MSRSB_EINVAL and "neighbourhood" in str(e.value)
    h = M.msrsb_setup(A, g, M.opts(smoother=B.MSRSB_SMOOTH_L1JAC))
    h.destroy()


@pytest.mark.parametrize("prec", [0, 1])
def test_paper_rough_grid_mpfa_case(M, prec):
    """The 2D MPFA-O test of Sec. 3.2 (100 x 100 rough cells on 20 m x 150 m,
    tensor [[100, 25], [25, 100]], 5 x 5-cell blocks, ILU(0) post-smoothing):
    GMRES and Richardson to 1e-8 within +-1 of the oracle's counts (line-block
    order on both sides), and ILU(0) alone does not converge in 150 Richardson
    iterations (as the paper reports)."""
    from synth.darcy import darcy_2d_perturbed_case
    B = M.msrsb
    c = darcy_2d_perturbed_case()
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    basis = dict(tol=1e-3, n_it=10, max_iter=100)
    ref = O.setup_scalar(Ah, c["dims"], c["H"], **basis)
    b = torch.as_tensor(c["b"], device="cuda")
    for kry, solver in ((B.MSRSB_GMRES, O.gmres_right), (B.MSRSB_RICHARDSON, O.richardson)):
        _, its_ref, _, _ = solver(Ah, c["b"], ref["tl"].apply, rtol=1e-8, maxit=300)
        h = M.msrsb_setup(A, g, M.opts(krylov=kry, prec=prec, **basis))
        r = h.solve(b, rtol=1e-8, maxit=300)
        x = r["x"].cpu().numpy()
        assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"])
        assert abs(r["iters"] - its_ref) <= 1, (kry, r["iters"], its_ref)
        h.destroy()
    h = M.msrsb_setup(A, g, M.opts(krylov=B.MSRSB_RICHARDSON, no_coarse=1, prec=prec, **basis))
    r = h.solve(b, rtol=1e-8, maxit=150, raise_on_noconv=False)
    assert r["iters"] == 150 and r["relres"] > 1e-8
    h.destroy()
