"""The differentiable two-point flux forward model of the adjoint module, on
the CPU (no GPU, no MsRSB): its matrix and right-hand side equal the
generator's two-point flux system, and torch autograd through it with a dense
direct solve gives the oracle's hand-derived adjoint gradient of a pressure
misfit with respect to log-permeability."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import msrsb as O  # noqa: E402
from synth.darcy import tpfa  # noqa: E402
from paper_1912_06934_gb300.adjoint import tpfa_darcy, tpfa_pattern  # noqa: E402


def _grid(logk, dims):
    # flat order x fastest -> array indexed [x, y, z]
    return np.asarray(logk).reshape(dims[::-1]).transpose(tuple(range(len(dims)))[::-1])


@pytest.mark.parametrize("dims", [(5, 4, 3), (6, 5)])
def test_forward_model_matches_the_generator(dims):
    rng = np.random.default_rng(11)
    n = int(np.prod(dims))
    logk = rng.standard_normal(n)
    pat = tpfa_pattern(dims, device="cpu")
    vals, b = tpfa_darcy(torch.as_tensor(logk), pat)
    A = sp.csr_matrix((vals.numpy(), pat["colidx"].numpy(), pat["rowptr"].numpy()), shape=(n, n))
    d = len(dims)
    K = np.exp(_grid(logk, dims))[..., None, None] * np.eye(d)
    ip, ix, dv, bg = tpfa(K, bc={(0, 0): ("D", 1.0), (0, 1): ("D", 0.0)})
    G = sp.csr_matrix((dv, ix, ip), shape=(n, n))
    assert abs(A - G).max() <= 1e-13 * abs(G).max()
    assert np.abs(b.numpy() - bg).max() <= 1e-13 * np.abs(bg).max()


def test_autograd_through_the_forward_model_gives_the_adjoint_gradient():
    dims = (4, 3, 2)
    n = int(np.prod(dims))
    rng = np.random.default_rng(5)
    logk = rng.standard_normal(n)
    obs = np.array([1, 7, 12, 20])
    p_obs = rng.uniform(0.2, 0.8, size=len(obs))
    pat = tpfa_pattern(dims, device="cpu")
    th = torch.as_tensor(logk).requires_grad_(True)
    vals, b = tpfa_darcy(th, pat)
    rows = torch.repeat_interleave(torch.arange(n), torch.diff(pat["rowptr"].long()))
    A = torch.zeros(n, n, dtype=torch.float64).index_put((rows, pat["colidx"].long()), vals, accumulate=True)
    p = torch.linalg.solve(A, b)
    J = ((p[torch.as_tensor(obs)] - torch.as_tensor(p_obs)) ** 2).sum()
    J.backward()
    J_ref, g_ref, p_ref = O.tpfa_objective_gradient(dims, logk, obs, p_obs)
    assert np.abs(p.detach().numpy() - p_ref).max() <= 1e-12
    assert abs(float(J.detach()) - J_ref) <= 1e-12 * abs(J_ref)
    assert np.linalg.norm(th.grad.numpy() - g_ref) <= 1e-10 * np.linalg.norm(g_ref)
