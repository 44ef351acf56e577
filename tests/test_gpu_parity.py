"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer work (partition, pattern, skeleton) must match bit for bit; the filter
is computed in the same order on both sides and must match exactly; P within
1e-11 max-abs in FP64 and 1e-5 in FP32 (entries lie in [0, 1]); A_c within
1e-12 of its largest entry; the preconditioner apply within 1e-10 relative;
Krylov solves to relative residual 1e-8 with iteration counts within +-1.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import darcy_2d_case, darcy_3d_case  # noqa: E402
from synth.elastic import elastic_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu

P_TOL64 = 1e-11
P_TOL32 = 1e-5


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _csr(c):
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    A.sort_indices()
    return A


def _gpu_P(p_ids, p_val, nc):
    ids = p_ids.cpu().numpy()
    vals = p_val.cpu().numpy().astype(np.float64)
    rows, slots = np.nonzero(ids >= 0)
    return sp.csr_matrix((vals[rows, slots], (rows, ids[rows, slots])), shape=(ids.shape[0], nc))


def _pattern_sets(p_ids):
    ids = p_ids.cpu().numpy()
    return [tuple(sorted(r[r >= 0])) for r in ids]


# ---------------- partition (bit exact) ----------------

@pytest.mark.parametrize("dims,H,cen", [((64, 64), (8, 8), 0), ((24, 24, 24), (8, 8, 8), 0),
                                        ((20, 18, 13), (8, 6, 4), 0), ((13, 13, 13), (6, 6, 6), 1),
                                        ((11, 9), (4, 3), 1), ((5, 3, 2), (8, 8, 8), 0)])
def test_partition_bitexact(M, dims, H, cen):
    g = M.grid(dims, H, centering=cen)
    part, cnode, p_ids, skel = M.msrsb_partition(g)
    ref = O.partition(dims, H, cen)
    assert np.array_equal(part.cpu().numpy(), ref["part"])
    assert np.array_equal(cnode.cpu().numpy(), ref["cnode"])
    assert np.array_equal(skel.cpu().numpy().astype(bool), ref["skel"])
    pat = ref["pat"]
    want = [tuple(pat.indices[pat.indptr[i]:pat.indptr[i + 1]]) for i in range(pat.shape[0])]
    assert _pattern_sets(p_ids) == want
    # colour slots: coarse node J sits in slot sum_d (J_d mod 2) 2^d in every row
    ids = p_ids.cpu().numpy()
    nb = ref["nb"]
    r, s = np.nonzero(ids >= 0)
    J = ids[r, s]
    col = np.zeros_like(J)
    rem = J.copy()
    for d in range(len(dims)):
        col |= (rem % nb[d] % 2) << d
        rem //= nb[d]
    assert np.array_equal(col, s)


# ---------------- filter (same order of operations -> exact) ----------------

def test_filter_exact_scalar(M):
    c = darcy_3d_case(n=16)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    ahat, nz = M.msrsb_filter(A)
    ref = O.mmatrix_filter(_csr(c))
    assert np.array_equal(ahat.cpu().numpy(), ref.data)
    assert nz == 0


def test_filter_exact_sdc(M):
    c = elastic_3d_case(ne=6, H=3)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=3)
    comps = O.sdc_blocks(c["indptr"], c["indices"], c["data"])
    nfixed = int(c["fixed"].sum())
    for l in range(3):
        ahat, nz = M.msrsb_filter(A, comp=l)
        ref = O.mmatrix_filter(comps[l])
        assert np.array_equal(ahat.cpu().numpy(), ref.data)
        assert nz == nfixed  # fixed nodes keep only their diagonal


# ---------------- basis ----------------

def _basis_case(M, c, prec, iters, tol=0.0, n_it=10):
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    ahat, _ = M.msrsb_filter(A)
    Ah = M.Mat(A.rowptr, A.colidx, ahat)
    g = M.grid(c["dims"], c["H"])
    part, cnode, p_ids, skel = M.msrsb_partition(g)
    W = p_ids.shape[1]
    dt = torch.float64 if prec == 0 else torch.float32
    P = ((p_ids >= 0) & (p_ids == part[:, None].to(torch.int32))).to(dt).contiguous()
    it, e = M.msrsb_build_basis(Ah, p_ids, skel, W, M.basis_opts(tol=tol, n_it=n_it, max_iter=iters), prec, P)
    return p_ids, P, it, e


@pytest.mark.parametrize("case", ["2d64", "3d24", "3d_ragged"])
def test_basis_fp64_matches_oracle(M, case):
    c = {"2d64": lambda: darcy_2d_case(),
         "3d24": lambda: darcy_3d_case(n=24),
         "3d_ragged": lambda: darcy_3d_case(dims=(20, 18, 13), H=(8, 6, 4))}[case]()
    iters = 40
    p_ids, P, it, e = _basis_case(M, c, 0, iters)
    ref = O.partition(c["dims"], c["H"], 0)
    Ah = O.mmatrix_filter(_csr(c))
    vals, k, e_ref, _ = O.enhanced_msrsb(Ah, ref["pat"], O.indicator(ref["part"], ref["pat"]), ref["skel"],
                                         tol=0.0, n_it=10, max_iter=iters)
    assert it == k == iters
    diff = np.abs(_gpu_P(p_ids, P, ref["nc"]).toarray() - O.as_matrix(vals, ref["pat"]).toarray()).max()
    assert diff <= P_TOL64
    assert abs(e - e_ref) <= 1e-12


def test_basis_fp32_matches_oracle(M):
    c = darcy_3d_case(n=24)
    p_ids, P, it, e = _basis_case(M, c, 1, 100)
    ref = O.partition(c["dims"], c["H"], 0)
    Ah = O.mmatrix_filter(_csr(c))
    vals, k, e_ref, _ = O.enhanced_msrsb(Ah, ref["pat"], O.indicator(ref["part"], ref["pat"]), ref["skel"],
                                         tol=0.0, n_it=10, max_iter=100)
    diff = np.abs(_gpu_P(p_ids, P, ref["nc"]).toarray() - O.as_matrix(vals, ref["pat"]).toarray()).max()
    assert diff <= P_TOL32


def test_basis_tolerance_stop_matches_oracle(M):
    # Alg. 1 stopping rule: check when k mod n_it == 0, stop once e_it <= tol
    c = darcy_2d_case(n=48, H=8)
    p_ids, P, it, e = _basis_case(M, c, 0, 500, tol=1e-3, n_it=7)
    ref = O.partition(c["dims"], c["H"], 0)
    vals, k, e_ref, hist = O.enhanced_msrsb(O.mmatrix_filter(_csr(c)), ref["pat"],
                                            O.indicator(ref["part"], ref["pat"]), ref["skel"],
                                            tol=1e-3, n_it=7, max_iter=500)
    assert it == k and k < 500 and (k - 1) % 7 == 0
    assert abs(e - e_ref) <= 1e-12 and e <= 1e-3


def test_basis_one_pass_at_full_size(M):
    # 64^3 (the benchmark's grid): the GPU's pass k+1 equals the oracle's single
    # pass applied to the GPU's own pass-k basis
    c = darcy_3d_case(n=64)
    k = 5
    p_ids, Pk, _, _ = _basis_case(M, c, 0, k)
    _, Pk1, _, _ = _basis_case(M, c, 0, k + 1)
    ref = O.partition(c["dims"], c["H"], 0)
    Ah = O.mmatrix_filter(_csr(c))
    Pg = _gpu_P(p_ids, Pk, ref["nc"])
    Pg.sort_indices()
    # re-express on the oracle pattern (explicit zeros kept)
    vals_k = np.asarray(Pg[np.repeat(np.arange(Pg.shape[0]), np.diff(ref["pat"].indptr)), ref["pat"].indices]).ravel()
    nxt, _ = O.smoothing_pass(Ah, ref["pat"], vals_k, O.inverse_diagonal(Ah), 2.0 / 3.0)
    Pn = _gpu_P(p_ids, Pk1, ref["nc"])
    got = np.asarray(Pn[np.repeat(np.arange(Pn.shape[0]), np.diff(ref["pat"].indptr)), ref["pat"].indices]).ravel()
    assert np.abs(got - nxt).max() <= 1e-13
    # invariants of the full-size basis
    rs = np.asarray(Pn.sum(axis=1)).ravel()
    assert np.abs(rs - 1).max() <= 1e-14 and got.min() >= 0 and got.max() <= 1 + 1e-15


# ---------------- Galerkin ----------------

def _coarse_stencil_pattern(nb):
    """Brute force: coarse nodes L with |L_d - J_d| <= 1 on every axis, per
    row J in ascending order (x fastest)."""
    coords = np.indices(nb[::-1]).reshape(len(nb), -1)[::-1].T  # (nc, d), x fastest
    rowptr, cols = [0], []
    for J in range(len(coords)):
        near = np.flatnonzero(np.all(np.abs(coords - coords[J]) <= 1, axis=1))
        cols.extend(near.tolist())
        rowptr.append(len(cols))
    return np.array(rowptr), np.array(cols)


@pytest.mark.parametrize("case", ["darcy3d", "darcy2d", "elastic"])
def test_coarse_op_matches_oracle(M, case):
    """msrsb_coarse_op's block CSR: pattern bit-exact against the brute-force
    coarse stencil, values within 1e-12 of the oracle's P^T A P."""
    if case == "darcy3d":
        c = darcy_3d_case(dims=(40, 24, 16), H=8)
    elif case == "darcy2d":
        c = darcy_2d_case(n=40, H=8)
    else:
        c = elastic_3d_case(ne=10, H=4)
    bd = c["ncomp"]
    g = M.grid(c["dims"], c["H"], centering=c["centering"], ncomp=bd)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=bd)
    o = M.opts(tol=0.0, max_iter=20, **(dict(smoother=M.msrsb.MSRSB_SMOOTH_GS, pre=1, post=1) if bd == 3 else {}))
    h = M.msrsb_setup(A, g, o)
    p_ids, P, _ = h.get_setup()
    h.destroy()
    part = O.partition(c["dims"], c["H"], c["centering"])
    nc, nb = part["nc"], part["nb"]
    rowptr, colidx, val = M.msrsb_coarse_op(A, g, p_ids, P, 0)
    rp, ci = _coarse_stencil_pattern(nb)
    assert np.array_equal(rowptr.cpu().numpy(), rp)
    assert np.array_equal(colidx.cpu().numpy(), ci)
    assert int(np.prod([3 * k - 2 for k in nb])) == len(ci)
    Acg = sp.bsr_matrix((val.cpu().numpy(), ci, rp), shape=(nc * bd, nc * bd)).toarray()
    if bd == 1:
        ref = O.galerkin(_csr(c), _gpu_P(p_ids, P[0], nc)).toarray()
    else:
        Pb = O.block_prolongation([_gpu_P(p_ids, P[l], nc) for l in range(3)])
        ref = O.galerkin(O.bsr_to_csr(c["indptr"], c["indices"], c["data"]), Pb).toarray()
    assert np.abs(Acg - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("case", ["2d64", "3d24", "ragged", "one_plane", "elastic12", "wide_planes"])
def test_coarse_solver_is_exact(M, case):
    """The block LU over coarse planes applies A_c^-1 exactly: with no
    smoother, one application is z = P A_c^-1 P^T v. w = A_c^-1 P^T v is
    recovered from z by least squares (P has full column rank; normal
    equations with the well-conditioned P^T P) and its
    backward error |A_c w - P^T v| / (|A_c| |w|) must be at rounding level
    (1e-13); against LAPACK's LU with partial pivoting (scipy) on the GPU's own
    A_c and P, z agrees within the forward-error bound of a backward-stable
    solve, 100 kappa(A_c) u (at least 1e-10). A_c itself is checked against
    the oracle above. Geometries: 2D lines, 3D planes, a ragged coarse grid, a
    single plane, 3x3 blocks, and planes of 256 nodes as in the 128^3
    workload."""
    import scipy.linalg as sla
    B = M.msrsb
    if case == "2d64":
        c = darcy_2d_case(n=64, H=8)
    elif case == "3d24":
        c = darcy_3d_case(n=24, H=8)
    elif case == "ragged":
        c = darcy_3d_case(dims=(40, 24, 21), H=8)
    elif case == "one_plane":
        c = darcy_3d_case(dims=(32, 32, 8), H=8)
    elif case == "elastic12":
        c = elastic_3d_case(ne=12, H=4)
    else:
        c = darcy_3d_case(dims=(128, 128, 24), H=8)
    bd = c["ncomp"]
    g = M.grid(c["dims"], c["H"], centering=c["centering"], ncomp=bd)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=bd)
    kw = dict(smoother=B.MSRSB_SMOOTH_NONE, pre=0, post=0, tol=0.0, max_iter=3)
    if bd == 3:
        kw["krylov"] = B.MSRSB_PCG
    h = M.msrsb_setup(A, g, M.opts(**kw))
    p_ids, P, Ac = h.get_setup()
    nc = h.info()["nc"]
    if bd == 1:
        Pg = _gpu_P(p_ids, P[0], nc)
    else:
        Pg = O.block_prolongation([_gpu_P(p_ids, P[l], nc) for l in range(3)])
    v = np.random.default_rng(8).standard_normal(Pg.shape[0])
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    h.destroy()
    Acd = Ac.cpu().numpy()
    vc = Pg.T @ v
    Pc = sp.csr_matrix(Pg)
    w = sp.linalg.spsolve((Pc.T @ Pc).tocsc(), Pc.T @ z)  # P^T P: SPD, well conditioned
    assert np.linalg.norm(Acd @ w - vc) <= 1e-13 * np.linalg.norm(Acd, 2) * np.linalg.norm(w)
    zr = Pg @ sla.lu_solve(sla.lu_factor(Acd), vc)
    kappa = np.linalg.cond(Acd)
    assert np.linalg.norm(z - zr) <= max(1e-10, 100 * kappa * 2.2e-16) * np.linalg.norm(zr)


# ---------------- set-up, apply, solve ----------------

def _setup(M, c, prec=0, tol=0.0, max_iter=30, bdim=1, **kw):
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=bdim)
    g = M.grid(c["dims"], c["H"], centering=c["centering"], ncomp=c["ncomp"])
    o = M.opts(tol=tol, max_iter=max_iter, prec=prec, **kw)
    return A, M.msrsb_setup(A, g, o)


def test_setup_apply_matches_oracle_scalar(M):
    c = darcy_3d_case(n=24)
    A, h = _setup(M, c)
    p_ids, p_val, Ac = h.get_setup()
    ref = O.setup_scalar(_csr(c), c["dims"], c["H"], tol=0.0, max_iter=30)
    nc = ref["part"]["nc"]
    assert np.abs(_gpu_P(p_ids, p_val[0], nc).toarray() - ref["P"].toarray()).max() <= P_TOL64
    Acr = ref["tl"].Ac.toarray()
    assert np.abs(Ac.cpu().numpy() - Acr).max() <= 1e-12 * np.abs(Acr).max()
    v = np.random.default_rng(3).standard_normal(A.nrows)
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = ref["tl"].apply(v)
    assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr)
    h.destroy()


def test_gmres_matches_oracle_2d(M):
    c = darcy_2d_case()
    A, h = _setup(M, c, tol=1e-3, max_iter=100)
    b = torch.as_tensor(c["b"], device="cuda")
    res = h.solve(b, rtol=1e-8, maxit=300, hist=True)
    Ah = _csr(c)
    ref = O.setup_scalar(Ah, c["dims"], c["H"], tol=1e-3, max_iter=100)
    assert h.info()["basis_iters"] == ref["iters"]
    xo, it_o, rr_o, hist_o = O.gmres_right(Ah, c["b"], ref["tl"].apply, rtol=1e-8, maxit=300)
    x = res["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"])
    assert abs(res["iters"] - it_o) <= 1
    assert np.allclose(res["hist"][1:6], hist_o[:5], rtol=1e-6)
    h.destroy()


def test_gmres_matches_oracle_3d(M):
    c = darcy_3d_case(n=32)
    A, h = _setup(M, c, tol=1e-3, max_iter=100)
    res = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=300)
    Ah = _csr(c)
    ref = O.setup_scalar(Ah, c["dims"], c["H"], tol=1e-3, max_iter=100)
    xo, it_o, rr_o, _ = O.gmres_right(Ah, c["b"], ref["tl"].apply, rtol=1e-8, maxit=300)
    x = res["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"])
    assert abs(res["iters"] - it_o) <= 1
    h.destroy()


def test_mixed_precision_solve(M):
    c = darcy_3d_case(n=32)
    A, h = _setup(M, c, prec=1, tol=1e-3, max_iter=100)
    res = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=300)
    Ah = _csr(c)
    x = res["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"])
    p_ids, p_val, _ = h.get_setup()
    ref = O.setup_scalar(Ah, c["dims"], c["H"], tol=1e-3, max_iter=100)
    nc = ref["part"]["nc"]
    assert np.abs(_gpu_P(p_ids, p_val[0], nc).toarray() - ref["P"].toarray()).max() <= P_TOL32
    h.destroy()


def test_pcg_elastic_matches_oracle(M):
    c = elastic_3d_case(ne=12, H=6)
    from paper_1912_06934_gb300 import msrsb as B
    A, h = _setup(M, c, bdim=3, tol=1e-3, max_iter=100, smoother=B.MSRSB_SMOOTH_GS, pre=1, post=1,
                  krylov=B.MSRSB_PCG)
    res = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=500)
    ref = O.setup_elastic(c["indptr"], c["indices"], c["data"], c["dims"], c["H"], tol=1e-3, max_iter=100)
    p_ids, p_val, Ac = h.get_setup()
    nc = ref["part"]["nc"]
    for l in range(3):
        Pl = O.as_matrix(ref["comps"][l][0], ref["part"]["pat"]).toarray()
        assert np.abs(_gpu_P(p_ids, p_val[l], nc).toarray() - Pl).max() <= P_TOL64
    Acr = ref["tl"].Ac.toarray()
    assert np.abs(Ac.cpu().numpy() - Acr).max() <= 1e-12 * np.abs(Acr).max()
    v = np.random.default_rng(5).standard_normal(3 * c["indptr"].shape[0] - 3)
    z = h.apply(torch.as_tensor(v, device="cuda")).cpu().numpy()
    zr = ref["tl"].apply(v)
    assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr)
    xo, it_o, rr_o, _ = O.pcg(ref["A"], c["b"], ref["tl"].apply, rtol=1e-8, maxit=500)
    x = res["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - ref["A"] @ x) <= 1e-8 * np.linalg.norm(c["b"])
    assert abs(res["iters"] - it_o) <= 1
    h.destroy()


def test_solve_host_buffers(M):
    c = darcy_2d_case(n=32)
    g = M.grid(c["dims"], c["H"])
    o = M.opts(tol=1e-3, max_iter=50)
    x = np.zeros_like(c["b"])
    it, rr = M.msrsb_solve_host(c["indptr"], c["indices"], c["data"], 1, g, o, c["b"], x)
    Ah = _csr(c)
    assert np.linalg.norm(c["b"] - Ah @ x) <= 1e-8 * np.linalg.norm(c["b"]) and rr <= 1e-8 and it > 0


def test_errors_are_reported(M):
    c = darcy_2d_case(n=16)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid((16, 15), (4, 4))  # wrong size
    with pytest.raises(M.MsrsbError) as e:
        M.msrsb_setup(A, g, M.opts())
    assert e.value.status == 2
