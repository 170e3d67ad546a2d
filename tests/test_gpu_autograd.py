"""Differentiable solve u = solve(A(kappa), b) through the PSLR adjoint
(FGMRES on A^T preconditioned by pslr_apply_T, gradient on A's pattern by
pslr_grad_values), checked against central finite differences of the exact
loss and against the dense-LU gradient."""
import numpy as np
import pytest

from pslr_inputs import configs as C
from pslr_inputs import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build

    build.build()
    return torch.device("cuda:0")


def _problem():
    dims = (8, 7, 6)
    w = C.small_problem("kappa", dims, (2, 2, 2), factor=0, m=3, rank=8, K=3)
    kap = G.kappa_field(dims, 0.5, 0)
    return dims, w, kap


def test_gradients_match_dense_lu_and_finite_differences(dev):
    from paper_2002_00917_gb300 import autograd as AG

    dims, w, kap0 = _problem()
    A, sigma = w["A"], w["sigma"]
    b0, _ = G.uniform_rhs(A, 0)
    ut = torch.tensor(np.random.default_rng(1).uniform(-1, 1, A.n), device=dev)
    kappa = torch.tensor(kap0, device=dev, requires_grad=True)
    b = torch.tensor(b0, device=dev, requires_grad=True)
    vals = G.variable_kappa_values(dims, A, kappa, sigma, xp=torch)
    opts = dict(dims=w["dims"], splits=w["splits"], m=3, rank=8, rtol=1e-13, restart=80, maxit=4000)
    u = AG.solve(vals, b, A.rowptr, A.col, **opts)
    loss = torch.sum((u - ut) ** 2)
    loss.backward()
    gk = kappa.grad.cpu().numpy()
    gb = b.grad.cpu().numpy()

    # dense-LU reference (exact solves)
    utn = ut.cpu().numpy()

    def dense_loss(kv, bv):
        D = G.dense_from_csr(G.variable_kappa(dims, kv, sigma))
        return float(np.sum((np.linalg.solve(D, bv) - utn) ** 2))

    D = G.dense_from_csr(A)
    ud = np.linalg.solve(D, b0)
    lamd = np.linalg.solve(D.T, 2 * (ud - utn))
    np.testing.assert_allclose(gb, lamd, rtol=1e-7, atol=1e-9 * np.abs(lamd).max())
    np.testing.assert_allclose(u.detach().cpu().numpy(), ud, rtol=1e-9, atol=1e-10)
    # dense gradient w.r.t. kappa: chain rule through the assembly with torch on the CPU
    kc = torch.tensor(kap0, requires_grad=True)
    vc = G.variable_kappa_values(dims, A, kc, sigma, xp=torch)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    gA = torch.tensor(-lamd[rows] * ud[A.col])
    (vc * gA).sum().backward()
    np.testing.assert_allclose(gk, kc.grad.numpy(), rtol=1e-7, atol=1e-9 * np.abs(kc.grad.numpy()).max())
    # central finite differences of the exact loss, h = 1e-6, on seeded entries
    idx = np.random.default_rng(2).choice(A.n, 6, replace=False)
    for i in idx:
        h = 1e-6
        kp, km = kap0.copy(), kap0.copy()
        kp[i] += h
        km[i] -= h
        fd = (dense_loss(kp, b0) - dense_loss(km, b0)) / (2 * h)
        assert abs(fd - gk[i]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gk).max()), (i, fd, gk[i])
