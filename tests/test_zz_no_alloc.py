"""The allocation-free basis build (msrsb_build_basis_noalloc) against the
regular entry point, through the C ABI.

Some callers cannot allocate device memory (an external memory manager owns
the GPU, or the host loop must not take the allocator's locks); the variant
keeps its scratch in a static device array shared by all calls. This file is
collected last so that a run stopping at the first failure has already run
every other test; it must pass alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth.darcy import darcy_2d_case, darcy_3d_case  # noqa: E402

pytestmark = pytest.mark.gpu

P_TOL64 = 1e-11  # the tolerance the parity tests use for P in FP64
P_TOL32 = 1e-5


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def _inputs(M, c, prec):
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    ahat, _ = M.msrsb_filter(A)
    Ah = M.Mat(A.rowptr, A.colidx, ahat)
    part, cnode, p_ids, skel = M.msrsb_partition(M.grid(c["dims"], c["H"]))
    dt = torch.float64 if prec == 0 else torch.float32
    P0 = ((p_ids >= 0) & (p_ids == part[:, None].to(torch.int32))).to(dt).contiguous()
    return Ah, p_ids, skel, P0


def _compare(M, c, prec, tol, n_it, max_iter):
    Ah, p_ids, skel, P0 = _inputs(M, c, prec)
    W = p_ids.shape[1]
    bo = M.basis_opts(tol=tol, n_it=n_it, max_iter=max_iter)
    P_ref = P0.clone()
    it_ref, e_ref = M.msrsb_build_basis(Ah, p_ids, skel, W, bo, prec, P_ref)
    P_new = P0.clone()
    it_new, e_new = M.msrsb_build_basis_noalloc(Ah, p_ids, skel, W, bo, prec, P_new)
    torch.cuda.synchronize()
    bound = P_TOL64 if prec == 0 else P_TOL32
    assert it_new == it_ref
    assert abs(e_new - e_ref) <= bound
    assert (P_new - P_ref).abs().max().item() <= bound


def test_noalloc_matches_build_basis_two_calls_in_a_row(M):
    # first call stops early on the tolerance (its done flag stays in the
    # static scratch); the second call, larger and in 3D, must start clean
    _compare(M, darcy_2d_case(n=48, H=8), 0, tol=1e-3, n_it=7, max_iter=300)
    _compare(M, darcy_3d_case(n=24), 0, tol=0.0, n_it=10, max_iter=30)


def test_noalloc_fp32_two_calls_in_a_row(M):
    c = darcy_3d_case(n=20, H=4)
    _compare(M, c, 1, tol=0.0, n_it=10, max_iter=40)
    _compare(M, c, 1, tol=0.0, n_it=10, max_iter=40)


def test_noalloc_rejects_inputs_beyond_its_scratch(M):
    # 64^3 rows x 8 slots exceed n * W <= 2^20: refused before any device work
    c = darcy_3d_case(n=64)
    Ah, p_ids, skel, P0 = _inputs(M, c, 0)
    with pytest.raises(M.MsrsbError) as e:
        M.msrsb_build_basis_noalloc(Ah, p_ids, skel, 8, M.basis_opts(), 0, P0)
    assert e.value.status == 2 and "static scratch" in str(e.value)
