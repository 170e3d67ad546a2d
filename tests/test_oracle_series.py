"""Pins for the splitting, the power series and E_rr(m) (Sec. 3.1 and 3.2)."""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C

from conftest import dense_operators

CASES = [
    ("lap", (12, 10), (3, 2), 0),
    ("lap", (12, 10), (3, 2), 1),
    ("cd", (6, 6, 6), (3, 2, 1), 0),
    ("kappa", (5, 6, 4), (2, 3, 1), 0),
    ("lap", (6, 5, 4), (2, 2, 2), 1),
]


def _setup(kind, dims, splits, factor):
    o = O.from_workload(C.small_problem(kind, dims, splits, factor=factor, K=3))
    D = dense_operators(o, factor)
    # Sec. 3.1: E_s = (C0 - C) + F B^{-1} E = -C_g + F B^{-1} E, with B^{-1} the
    # local-factor solve B~^{-1}; the split Schur complement is then
    # S~ = C0~ - E_s (Eq. 3.1), which is S = C - F B^{-1} E (Eq. 2.2) for exact factors.
    Es = -D["Cg"] + D["F"] @ np.linalg.solve(D["Bt"], D["E"])
    S = D["C0t"] - Es
    return o, D, S, Es


def _columns(fn, q):
    return np.stack([fn(e) for e in np.eye(q)], axis=1)


@pytest.mark.parametrize("kind,dims,splits,factor", CASES)
def test_splitting_Es(kind, dims, splits, factor):
    o, D, S, Es = _setup(kind, dims, splits, factor)
    np.testing.assert_allclose(_columns(o.Es, o.q), Es, atol=1e-12)
    np.testing.assert_allclose(_columns(o.EsT, o.q), Es.T, atol=1e-12)
    if factor == 1:
        np.testing.assert_allclose(S, D["C"] - D["F"] @ np.linalg.solve(D["B"], D["E"]), atol=1e-12)


@pytest.mark.parametrize("kind,dims,splits,factor", CASES)
@pytest.mark.parametrize("m", [0, 1, 3, 5])
def test_series_closed_form(kind, dims, splits, factor, m):
    """Eq. 3.3 summed in closed form: sum_{i=0}^m N^i = (I - N^{m+1})(I - N)^{-1},
    N = C0^{-1} E_s; valid whenever I - N is nonsingular, even for rho(N) > 1."""
    o, D, S, Es = _setup(kind, dims, splits, factor)
    q = o.q
    C0i = np.linalg.inv(D["C0t"])
    N = C0i @ Es
    Pm = (np.eye(q) - np.linalg.matrix_power(N, m + 1)) @ np.linalg.inv(np.eye(q) - N) @ C0i
    got = _columns(lambda v: o.series(m, v), q)
    np.testing.assert_allclose(got, Pm, atol=1e-10 * np.abs(Pm).max())
    gotT = _columns(lambda v: o.seriesT(m, v), q)
    np.testing.assert_allclose(gotT, Pm.T, atol=1e-10 * np.abs(Pm).max())
    if m == 0:
        np.testing.assert_allclose(got, C0i, atol=1e-12)


@pytest.mark.parametrize("kind,dims,splits,factor", CASES)
@pytest.mark.parametrize("m", [0, 2, 3])
def test_theorem_Err(kind, dims, splits, factor, m):
    """Eq. 3.13-3.14 define E_rr(m) = I - S P_m; the theorem of Sec. 3.2.1 (Eq.
    3.19) states it equals (E_s C0^{-1})^{m+1} for any A."""
    o, D, S, Es = _setup(kind, dims, splits, factor)
    q = o.q
    Pm = _columns(lambda v: o.series(m, v), q)
    Err_def = np.eye(q) - S @ Pm
    Err_thm = np.linalg.matrix_power(Es @ np.linalg.inv(D["C0t"]), m + 1)
    got = _columns(lambda v: o.Err(m, v), q)
    scale = max(1.0, np.abs(Err_thm).max())
    np.testing.assert_allclose(got, Err_thm, atol=1e-10 * scale)
    np.testing.assert_allclose(Err_def, Err_thm, atol=1e-9 * scale)
    # Eq. 3.15: S^{-1} = P_m (I - E_rr(m))^{-1}
    np.testing.assert_allclose(Pm @ np.linalg.inv(np.eye(q) - got), np.linalg.inv(S),
                               atol=1e-8 * np.abs(np.linalg.inv(S)).max())


def test_lemma_spd_spectrum_inside_unit_interval():
    """Lemma of Sec. 3.1: A SPD => lambda(C0^{-1}E_s) < 1; with C diagonally
    dominant also > -1.  Unshifted Laplacian, exact local factors."""
    from pslr_inputs import generators as G
    A = G.shifted_laplacian((9, 8, 4), 0.0)
    o = O.Oracle(A, dims=(9, 8, 4), splits=(2, 2, 1), factor=1)
    D = dense_operators(o, 1)
    Es = _columns(o.Es, o.q)
    lam = np.linalg.eigvals(np.linalg.solve(D["C0"], Es))
    assert np.all(np.abs(lam.imag) < 1e-10)
    assert lam.real.max() < 1 and lam.real.min() > -1


@pytest.mark.parametrize("dims,splits,K", [((10, 9, 8), (2, 2, 1), 7), ((12, 11), (3, 2), 5), ((9, 8, 7), (1, 2, 2), 12)])
def test_eigenvalues_above_one_count_the_negative_eigenvalues_of_S(dims, splits, K):
    """Sec. 3.1-3.2 on an indefinite problem (the setting of the spectra the
    paper plots for a shifted 20^3 Laplacian): with exact local factors and C0
    positive definite, E_s C0^{-1} is similar to C0^{-1/2} E_s C0^{-1/2}, whose
    eigenvalues above 1 are those where S = C0 - E_s is negative (Sylvester's
    law of inertia); by Haynsworth's inertia additivity S has neg(A) - neg(B)
    negative eigenvalues.  The count is checked against dense eigenvalues of A
    and B, so a sign or block mistake in E_s, E, F or C_g fails it."""
    from pslr_inputs import generators as G
    nd = len(dims)
    d3 = tuple(dims) + (1,) * (3 - nd)
    s3 = tuple(splits) + (1,) * (3 - nd)
    sig, k = G.sigma_for_negative_count([G.laplacian_1d_eigs(d) for d in dims], K)
    A = G.shifted_laplacian(dims, sig)
    o = O.Oracle(A, dims=d3, splits=s3, factor=1)
    D = dense_operators(o, 1)
    assert np.linalg.eigvalsh(D["C0"]).min() > 0
    Es = _columns(o.Es, o.q)
    lam = np.linalg.eigvals(Es @ np.linalg.inv(D["C0"]))
    assert np.abs(lam.imag).max() < 1e-9
    neg_A = int((np.linalg.eigvalsh(G.dense_from_csr(A)) < 0).sum())
    neg_B = int((np.linalg.eigvalsh(D["B"]) < 0).sum())
    assert neg_A == k
    above = int((lam.real > 1).sum())
    assert above == neg_A - neg_B, (above, neg_A, neg_B)
    assert np.abs(lam.real - 1).min() > 1e-8  # no eigenvalue at the boundary


def test_proposition1_bound():
    """Proposition of Sec. 3.1 (Eq. 3.6): when ||C0^{-1}E_s|| < 1,
    ||S^{-1} - P_m|| <= ||C0^{-1}E_s||^{m+1} ||C0^{-1}|| / (1 - ||C0^{-1}E_s||)."""
    from pslr_inputs import generators as G
    A = G.shifted_laplacian((9, 8), -0.5)  # diagonally dominant: the norm is below 1
    o = O.Oracle(A, dims=(9, 8, 1), splits=(3, 2, 1), factor=1)
    D = dense_operators(o, 1)
    S = D["C"] - D["F"] @ np.linalg.solve(D["B"], D["E"])
    N = np.linalg.solve(D["C0"], D["C0"] - S)
    nN = np.linalg.norm(N, 2)
    assert nN < 1
    for m in (0, 1, 3):
        R = np.linalg.inv(S) - _columns(lambda v: o.series(m, v), o.q)
        bound = nN ** (m + 1) * np.linalg.norm(np.linalg.inv(D["C0"]), 2) / (1 - nN)
        assert np.linalg.norm(R, 2) <= bound * (1 + 1e-12)
