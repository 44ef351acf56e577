"""Ensembles (msrsb_solve_ensemble) and set-ups on concurrent streams.

Independent problems of uneven sizes, several right-hand sides each, run
concurrently on streams of their own: every result must equal, bit for bit,
what the problem's own msrsb_setup + msrsb_solve calls give (the kernels are
deterministic) and reach relative residual 1e-8, recomputed here in FP64; a
failing problem reports its own status without disturbing the others. The
coarse correction (Alg. 3 with no smoother) of a 48^3 problem, set up
sequentially and from concurrent host threads, must be the same bit for bit
and equal P A_c^-1 P^T v computed here from the GPU's own P and A_c.
"""
import threading

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from synth.darcy import darcy_2d_case, darcy_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _cases():
    return [darcy_3d_case(n=16, seed=40001), darcy_3d_case(dims=(20, 18, 13), H=(8, 6, 4), seed=40002),
            darcy_2d_case(n=48, H=8, seed=40003), darcy_3d_case(n=48, seed=40007), darcy_3d_case(n=24, seed=40004)]


def _problem(M, c, nrhs, seed):
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    rng = np.random.default_rng(seed)
    B = np.stack([c["b"]] + [Ah @ rng.standard_normal(len(c["b"])) for _ in range(nrhs - 1)])
    return A, g, torch.as_tensor(B, device="cuda"), torch.zeros(nrhs, len(c["b"]), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", [0, 1])
def test_ensemble_matches_individual_solves(M, prec):
    cases = _cases()
    o = M.opts(prec=prec, tol=1e-3, max_iter=100)
    probs = [_problem(M, c, 3, 50000 + i) for i, c in enumerate(cases)]
    out = M.msrsb_solve_ensemble(probs, o, rtol=1e-8, maxit=300, concurrency=3)
    for (A, g, B, X), (its, rr, st), c in zip(probs, out, cases):
        assert st == 0
        Ah = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
        h = M.msrsb_setup(A, g, o)
        for r in range(B.shape[0]):
            res = h.solve(B[r].contiguous(), rtol=1e-8, maxit=300)
            assert res["iters"] == its[r]
            assert torch.equal(res["x"], X[r])
            x = X[r].cpu().numpy()
            b = B[r].cpu().numpy()
            assert np.linalg.norm(b - Ah @ x) <= 1e-8 * np.linalg.norm(b)
            assert rr[r] <= 1e-8
        h.destroy()


def test_ensemble_reports_a_failing_problem(M):
    cases = _cases()[:3]
    o = M.opts(prec=1, tol=1e-3, max_iter=50)
    probs = [_problem(M, c, 2, 60000 + i) for i, c in enumerate(cases)]
    A, g, B, X = probs[1]
    probs[1] = (A, M.grid((5, 5, 5), (8, 8, 8)), B, X)  # grid does not match the operator
    with pytest.raises(M.MsrsbError) as ei:
        M.msrsb_solve_ensemble(probs, o, rtol=1e-8, maxit=300, concurrency=2)
    assert "problem 1" in str(ei.value)
    for i in (0, 2):  # the other problems still ran to completion
        Xi = probs[i][3]
        assert torch.isfinite(Xi).all() and Xi.abs().sum() > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_coarse_correction_concurrent_setups(M, prec):
    from paper_1912_06934_gb300 import msrsb as B
    c = darcy_3d_case(n=48, seed=40008)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    o = M.opts(prec=prec, tol=1e-3, max_iter=100, smoother=B.MSRSB_SMOOTH_NONE)
    v = torch.as_tensor(np.random.default_rng(9).standard_normal(len(c["b"])), device="cuda")

    def one(stream):
        with torch.cuda.stream(stream):
            h = M.msrsb_setup(A, g, o, stream=stream)
            ids, P, Ac = h.get_setup(stream=stream)
            z = h.apply(v, stream=stream)
            stream.synchronize()
            out = (ids.clone(), P[0].double().clone(), Ac.clone(), z.clone())
            h.destroy()
        return out

    ref = one(torch.cuda.current_stream())
    ids, P, Ac, z = [t.cpu().numpy() for t in ref]
    rows, slots = np.nonzero(ids >= 0)
    Pm = sp.csr_matrix((P[rows, slots], (rows, ids[rows, slots])), shape=(ids.shape[0], Ac.shape[0]))
    z_host = Pm @ np.linalg.solve(Ac, Pm.T @ v.cpu().numpy())
    # the mixed form prolongs in FP32: each z_i is a sum of at most 8 products
    # of non-negative weights (a partition of unity), relative error <= 8 u_32
    assert np.linalg.norm(z - z_host) <= (1e-8 if prec == 0 else 1e-6) * np.linalg.norm(z_host)
    results = [None] * 6
    streams = [torch.cuda.Stream() for _ in range(6)]

    def worker(t):
        results[t] = one(streams[t])

    for _ in range(2):
        ths = [threading.Thread(target=worker, args=(t,)) for t in range(6)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for r in results:
            assert torch.equal(r[2], ref[2]) and torch.equal(r[3], ref[3])
