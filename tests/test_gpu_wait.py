"""The bounded device-side wait: the coarse inverse's CTAs wait on a
publication counter with a wall-time and poll limit. A wait on a counter that
nothing raises must give up, report MSRSB_ETIMEOUT, and leave the context
usable (a set-up and solve right after it succeed)."""
import time

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from synth.darcy import darcy_2d_case  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    return M


def test_wait_gives_up_and_context_stays_usable(M):
    from paper_1912_06934_gb300 import msrsb as B
    t0 = time.perf_counter()
    assert M.msrsb_wait_selftest(20.0) == B.MSRSB_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    c = darcy_2d_case(n=32, H=4)
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    h = M.msrsb_setup(M.Mat.from_host(c["indptr"], c["indices"], c["data"]), M.grid(c["dims"], c["H"]),
                      M.opts(prec=0))
    r = h.solve(torch.as_tensor(c["b"], device="cuda"), rtol=1e-8, maxit=200)
    x = r["x"].cpu().numpy()
    assert np.linalg.norm(c["b"] - A @ x) <= 1e-8 * np.linalg.norm(c["b"])
    h.destroy()


def test_wait_selftest_rejects_bad_limits(M):
    from paper_1912_06934_gb300 import msrsb as B
    for lim in (0.0, -1.0, 5000.0):
        assert M.msrsb_wait_selftest(lim) == B.MSRSB_EINVAL
