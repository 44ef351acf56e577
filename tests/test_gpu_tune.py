"""The launch-shape autotuner of the restricted-smoothing pass (Alg. 1).

Every launch shape (1 or 2 lanes per row; 256 or 128 threads per CTA; 0, 2 or 3
operator entries loaded ahead, registers free or capped) must
give P bit for bit equal to the one-lane shape, in FP64 and FP32, for W = 8
(3D) and W = 4 (2D), on grids whose row count is not a multiple of a warp or a
CTA. In automatic mode a new size class is timed once, recorded in the table,
and the result is still bit for bit the one-lane result; the oracle pins the
result itself (FP64 within 1e-11).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import darcy_2d_case, darcy_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu

N_SHAPES = 6
SHAPES = [(1, 256, 0, 0), (1, 128, 0, 0), (2, 256, 0, 0), (1, 256, 2, 0), (1, 256, 2, 1), (1, 256, 3, 1)]


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    yield M
    M.msrsb_tune_mode(M.MSRSB_TUNE_AUTO)


def _basis(M, c, prec, iters, tol=0.0, n_it=10):
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    ahat, _ = M.msrsb_filter(A)
    Ah = M.Mat(A.rowptr, A.colidx, ahat)
    g = M.grid(c["dims"], c["H"])
    part, cnode, p_ids, skel = M.msrsb_partition(g)
    W = p_ids.shape[1]
    dt = torch.float64 if prec == 0 else torch.float32
    P = ((p_ids >= 0) & (p_ids == part[:, None].to(torch.int32))).to(dt).contiguous()
    it, e = M.msrsb_build_basis(Ah, p_ids, skel, W, M.basis_opts(tol=tol, n_it=n_it, max_iter=iters), prec, P)
    torch.cuda.synchronize()
    return p_ids, P, it, e


CASES = {
    "3d_ragged": lambda: darcy_3d_case(dims=(20, 18, 13), H=(8, 6, 4)),  # n = 4,680, W = 8
    "3d24": lambda: darcy_3d_case(n=24),                                 # n = 13,824, W = 8
    "2d_ragged": lambda: darcy_2d_case(n=45, H=8),                       # n = 2,025, W = 4
}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_every_shape_is_bit_identical(M, case, prec):
    c = CASES[case]()
    res = []
    try:
        for v in range(N_SHAPES):
            M.msrsb_tune_mode(v)
            p_ids, P, it, e = _basis(M, c, prec, 30)
            res.append((P.cpu().numpy().copy(), it, e))
    finally:
        M.msrsb_tune_mode(M.MSRSB_TUNE_AUTO)
    P0, it0, e0 = res[0]
    assert it0 == 30
    for v in range(1, N_SHAPES):
        P, it, e = res[v]
        assert it == it0
        assert e == e0, "shape %d changed e_it" % v
        assert np.array_equal(P.view(np.uint8), P0.view(np.uint8)), "shape %d changed P" % v


def test_tolerance_stop_is_shape_independent(M):
    # Alg. 1's stop (check when k mod n_it == 0) must land on the same pass
    c = darcy_2d_case(n=48, H=8)
    out = []
    try:
        for v in range(N_SHAPES):
            M.msrsb_tune_mode(v)
            _, P, it, e = _basis(M, c, 0, 500, tol=1e-3, n_it=7)
            out.append((it, e, P.cpu().numpy().copy()))
    finally:
        M.msrsb_tune_mode(M.MSRSB_TUNE_AUTO)
    assert all(o[0] == out[0][0] and o[1] == out[0][1] for o in out)
    assert all(np.array_equal(o[2], out[0][2]) for o in out)
    assert out[0][0] < 500 and out[0][1] <= 1e-3


def test_auto_mode_records_a_class_and_keeps_the_result(M):
    c = darcy_3d_case(n=24)
    M.msrsb_tune_mode(0)
    try:
        _, P_ref, it_ref, e_ref = _basis(M, c, 1, 40)
    finally:
        M.msrsb_tune_mode(M.MSRSB_TUNE_AUTO)
    M.msrsb_tune_reset()
    assert M.msrsb_tune_table() == []
    _, P, it, e = _basis(M, c, 1, 40)
    assert it == it_ref and e == e_ref
    assert torch.equal(P, P_ref)
    tab = M.msrsb_tune_table()
    assert len(tab) == 1
    t = tab[0]
    n = 24 ** 3
    assert t["kernel"] == M.MSRSB_TUNE_SMOOTH and t["value_bytes"] == 4 and t["W"] == 8
    assert t["n_log2"] == math.ceil(math.log2(n)) and t["device"] == torch.cuda.current_device()
    assert t["n_variants"] == N_SHAPES and 0 <= t["variant"] < N_SHAPES
    assert all(u > 0 and math.isfinite(u) for u in t["us"])
    assert t["us"][t["variant"]] == min(t["us"])
    assert (t["lanes"], t["threads"], t["ahead"], t["capped"]) == SHAPES[t["variant"]]
    # a second loop of the same class reuses the entry (no new row, same result)
    _, P2, _, _ = _basis(M, c, 1, 40)
    assert torch.equal(P2, P_ref)
    assert len(M.msrsb_tune_table()) == 1
    # a loop too short to time every shape records nothing
    M.msrsb_tune_reset()
    _basis(M, c, 1, 3 * N_SHAPES + 3 * N_SHAPES // 2 - 1)
    assert M.msrsb_tune_table() == []


def test_auto_mode_matches_the_oracle(M):
    c = darcy_3d_case(dims=(20, 18, 13), H=(8, 6, 4))
    M.msrsb_tune_reset()
    p_ids, P, it, e = _basis(M, c, 0, 40)
    assert len(M.msrsb_tune_table()) == 1
    ref = O.partition(c["dims"], c["H"], 0)
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    A.sort_indices()
    vals, k, e_ref, _ = O.enhanced_msrsb(O.mmatrix_filter(A), ref["pat"], O.indicator(ref["part"], ref["pat"]),
                                         ref["skel"], tol=0.0, n_it=10, max_iter=40)
    ids = p_ids.cpu().numpy()
    pv = P.cpu().numpy()
    rows, slots = np.nonzero(ids >= 0)
    Pg = sp.csr_matrix((pv[rows, slots], (rows, ids[rows, slots])), shape=(ids.shape[0], ref["nc"]))
    assert it == k == 40
    assert np.abs(Pg.toarray() - O.as_matrix(vals, ref["pat"]).toarray()).max() <= 1e-11


def test_bad_mode_is_refused(M):
    for bad in (-2, N_SHAPES, 99):
        with pytest.raises(M.MsrsbError):
            M.msrsb_tune_mode(bad)
    M.msrsb_tune_mode(M.MSRSB_TUNE_AUTO)
