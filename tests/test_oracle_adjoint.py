"""The adjoint used for differentiation, on the oracle: for A u = b and
L = ||u - u_t||^2, lambda = A^{-T} dL/du and dL/da_ij = -lambda_i u_j; checked
against the closed form d(A^{-1}b)/da_ij = -A^{-1} e_i e_j^T A^{-1} b with
LAPACK solves, with FGMRES preconditioned by Algorithm 3 and by its transpose."""
import numpy as np

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G


def test_adjoint_gradient_matches_dense_formula():
    w = C.small_problem("kappa", (7, 6, 5), (2, 2, 1), factor=0, m=3, rank=6, K=3)
    A = w["A"]
    o = O.from_workload(w)
    o.build_lowrank(3, 6, seed=0)
    b, _ = G.uniform_rhs(A, 0)
    ut = np.random.default_rng(1).uniform(-1, 1, A.n)
    u, its, rel, st = o.fgmres(b, rtol=1e-13, restart=80, maxit=3000)
    assert st == O.OK
    gu = 2 * (u - ut)
    lam, its2, rel2, st2 = o.fgmres(gu, rtol=1e-13, restart=80, maxit=3000, transpose=True)
    assert st2 == O.OK
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    grad = -lam[rows] * u[A.col]
    D = G.dense_from_csr(A)
    ud = np.linalg.solve(D, b)
    lamd = np.linalg.solve(D.T, 2 * (ud - ut))
    gradd = -lamd[rows] * ud[A.col]
    np.testing.assert_allclose(lam, lamd, rtol=1e-8, atol=1e-10 * np.abs(lamd).max())
    np.testing.assert_allclose(grad, gradd, rtol=1e-7, atol=1e-9 * np.abs(gradd).max())
    # the same derivative by central differences of the exact (dense) loss
    L = lambda M: float(np.sum((np.linalg.solve(M, b) - ut) ** 2))
    for k in (0, 17, 101, len(A.val) - 1):
        i, j = rows[k], A.col[k]
        h = 1e-6
        Mp, Mm = D.copy(), D.copy()
        Mp[i, j] += h
        Mm[i, j] -= h
        fd = (L(Mp) - L(Mm)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gradd).max())
