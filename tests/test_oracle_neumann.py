"""Pins for the oracle's classical Neumann polynomial (Sec. 1): the foil the
paper contrasts PSLR with, S^{-1} ~ omega [I + N + ... + N^m] D^{-1},
N = I - omega D^{-1} S, with D = C0 and S = C0~ - E_s (Eq. 3.1)."""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

from conftest import dense_operators

CASES = [
    ("lap", (12, 10), (3, 2), 0),
    ("lap", (12, 10), (3, 2), 1),
    ("cd", (6, 6, 6), (3, 2, 1), 0),
    ("kappa", (5, 6, 4), (2, 3, 1), 0),
]


def _setup(kind, dims, splits, factor, K=3):
    w = C.small_problem(kind, dims, splits, factor=factor, K=K)
    o = O.from_workload(w)
    D = dense_operators(o, factor)
    Es = -D["Cg"] + D["F"] @ np.linalg.solve(D["Bt"], D["E"])
    S = D["C0t"] - Es
    return w, o, D, S


def _columns(fn, q):
    return np.stack([fn(e) for e in np.eye(q)], axis=1)


def _dense_series(D, S, m, omega):
    """omega sum_{i=0}^{m} N^i D^{-1}, N = I - omega D^{-1} S, by repeated products."""
    q = S.shape[0]
    Di = np.linalg.inv(D["C0t"])
    N = np.eye(q) - omega * Di @ S
    acc, P = np.zeros((q, q)), np.eye(q)
    for _ in range(m + 1):
        acc += P
        P = P @ N
    return omega * acc @ Di, N


@pytest.mark.parametrize("kind,dims,splits,factor", CASES)
@pytest.mark.parametrize("m,omega", [(0, 0.8), (2, 0.6), (3, 1.0), (5, 1.3)])
def test_neumann_series_dense(kind, dims, splits, factor, m, omega):
    """The series and its transpose against the dense sum."""
    w, o, D, S = _setup(kind, dims, splits, factor)
    Y, _ = _dense_series(D, S, m, omega)
    got = _columns(lambda v: o.neumann_series(m, omega, v), o.q)
    np.testing.assert_allclose(got, Y, atol=1e-10 * np.abs(Y).max())
    gotT = _columns(lambda v: o.neumann_series(m, omega, v, transpose=True), o.q)
    np.testing.assert_allclose(gotT, Y.T, atol=1e-10 * np.abs(Y).max())


@pytest.mark.parametrize("kind,dims,splits,factor", CASES)
@pytest.mark.parametrize("m", [0, 3])
def test_omega_one_is_the_power_series(kind, dims, splits, factor, m):
    """At omega = 1, N = I - D^{-1}(C0 - E_s) = C0^{-1} E_s: the polynomial is
    the method's own series P_m (Eq. 3.3), and the foil's apply is Algorithm 3
    with no low-rank term (the paper's r = 0 case)."""
    w, o, D, S = _setup(kind, dims, splits, factor)
    rng = np.random.default_rng(2)
    t = rng.uniform(-1, 1, o.q)
    a, b = o.neumann_series(m, 1.0, t), o.series(m, t)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    o.set_lowrank(m, None, None)
    rhs = rng.uniform(-1, 1, o.n)
    za, zb = o.neumann_apply(m, 1.0, rhs), o.apply(rhs)
    assert np.linalg.norm(za - zb) <= 1e-12 * np.linalg.norm(zb)


@pytest.mark.parametrize("kind,dims,splits,factor", CASES[:3])
def test_neumann_apply_block_elimination(kind, dims, splits, factor):
    """The apply is the block elimination of Eq. 2.2 with the polynomial as the
    Schur complement inverse (dense, reordered numbering), both directions."""
    w, o, D, S = _setup(kind, dims, splits, factor)
    m, omega = 3, 0.7
    Y, _ = _dense_series(D, S, m, omega)
    Bi = np.linalg.inv(D["Bt"])
    Minv = np.block([[Bi + Bi @ D["E"] @ Y @ D["F"] @ Bi, -Bi @ D["E"] @ Y], [-Y @ D["F"] @ Bi, Y]])
    perm = o.maps()[2]
    rng = np.random.default_rng(5)
    for tr in (False, True):
        b = rng.uniform(-1, 1, o.n)
        Mx = Minv.T if tr else Minv
        zr = Mx @ b[perm]
        z = np.empty(o.n)
        z[perm] = zr
        got = o.neumann_apply(m, omega, b, transpose=tr)
        assert np.linalg.norm(got - z) <= 1e-11 * np.linalg.norm(z), tr


def test_transpose_by_inner_products():
    """<M^{-1} u, v> = <u, M^{-T} v> on a 3D problem with ILU(0) factors."""
    w = C.small_problem("cd", (10, 9, 8), (2, 2, 2), factor=0, K=2)
    o = O.from_workload(w)
    rng = np.random.default_rng(3)
    u, v = rng.uniform(-1, 1, o.n), rng.uniform(-1, 1, o.n)
    for m, omega in ((2, 0.5), (4, 1.2)):
        a = o.neumann_apply(m, omega, u) @ v
        b = u @ o.neumann_apply(m, omega, v, transpose=True)
        assert abs(a - b) <= 1e-13 * (abs(a) + abs(b)), (m, omega)


def _spd_exact():
    """An SPD 2D Laplacian (no shift) with exact local LU: rho(N) < 1 for
    0 < omega <= 1 (Sec. 3.1's lemma puts the eigenvalues of D^{-1} S in (0, 2)
    here, where C is diagonally dominant)."""
    A = G.shifted_laplacian((14, 12), 0.0)
    w = dict(name="lap2d_spd", A=A, dims=(14, 12, 1), splits=(2, 2, 1), factor=1, m=0, rank=0)
    o = O.from_workload(w)
    D = dense_operators(o, 1)
    S = D["C"] - D["F"] @ np.linalg.solve(D["B"], D["E"])
    return A, o, D, S


def test_limit_is_the_exact_inverse_when_rho_below_one():
    """With exact factors and rho(N) < 1 the series converges to S^{-1}
    (S^{-1} = omega (I - N)^{-1} D^{-1}), so for m large enough the foil's
    apply is A^{-1}: FGMRES with it converges at once."""
    A, o, D, S = _spd_exact()
    omega = 0.9
    _, N = _dense_series(D, S, 0, omega)
    rho = np.abs(np.linalg.eigvals(N)).max()
    assert rho < 1.0
    m = int(np.ceil(np.log(1e-14) / np.log(rho)))
    b = np.random.default_rng(4).uniform(-1, 1, A.n)
    x = np.linalg.solve(G.dense_from_csr(A), b)
    z = o.neumann_apply(m, omega, b)
    assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x), (m, rho)
    o.set_neumann(m, omega)
    _, its, rel, st = o.fgmres(b, rtol=1e-10, restart=20, maxit=20)
    assert st == O.OK and its <= 2, (its, rel)


def test_more_terms_help_only_when_rho_below_one():
    """Sec. 1: the truncated series approaches S^{-1} as m grows only when
    rho(N) < 1.  With a shift that makes S indefinite, omega = 1 gives
    rho(N) > 1 and the error grows with m; on the SPD problem it falls."""
    A, o, D, S = _spd_exact()
    Si = np.linalg.inv(S)
    errs = [np.linalg.norm(_dense_series(D, S, m, 1.0)[0] - Si) for m in (2, 6, 12)]
    got = [np.linalg.norm(_columns(lambda v: o.neumann_series(m, 1.0, v), o.q) - Si) for m in (2, 6, 12)]
    np.testing.assert_allclose(got, errs, rtol=1e-8)
    assert got[0] > got[1] > got[2]
    # indefinite: 2D Laplacian shifted past 12 eigenvalues, exact factors
    w = C.small_problem("lap", (14, 12), (2, 2), factor=1, K=12)
    o2 = O.from_workload(w)
    D2 = dense_operators(o2, 1)
    S2 = D2["C"] - D2["F"] @ np.linalg.solve(D2["B"], D2["E"])
    _, N2 = _dense_series(D2, S2, 0, 1.0)
    assert np.abs(np.linalg.eigvals(N2)).max() > 1.0
    Si2 = np.linalg.inv(S2)
    got2 = [np.linalg.norm(_columns(lambda v: o2.neumann_series(m, 1.0, v), o2.q) - Si2) for m in (2, 6, 12)]
    assert got2[0] < got2[1] < got2[2]
