"""Pins for the synthetic problem generators (Section 4's test problems)."""
import numpy as np
import pytest

from pslr_inputs import configs as C
from pslr_inputs import generators as G


@pytest.mark.parametrize("N,shift,count", [
    # Section 4.1 (Laplacian test): 20, 69, 133 negative eigenvalues for
    # 32^3, 64^3, 128^3 at shifts .16, .08, .03; Table 4's text: 78 at 50^3, .14.
    (32, 0.16, 20), (64, 0.08, 69), (128, 0.03, 133), (50, 0.14, 78)])
def test_negative_counts_printed_in_paper(N, shift, count):
    lam = G._sum_spectrum([G.laplacian_1d_eigs(N)] * 3)
    assert int((lam < shift).sum()) == count


@pytest.mark.parametrize("dims", [(7,), (5, 4), (4, 3, 3)])
def test_closed_form_spectrum_matches_brute_force(dims):
    A = G.shifted_laplacian(dims, 0.0)
    ev = np.linalg.eigvalsh(G.dense_from_csr(A))
    lam = G._sum_spectrum([G.laplacian_1d_eigs(d) for d in dims])
    np.testing.assert_allclose(np.sort(ev), lam, atol=1e-12)


@pytest.mark.parametrize("dims", [(6, 6, 6), (5, 4, 3)])
def test_convdiff_closed_form_spectrum(dims):
    A = G.convection_diffusion(dims, 50.0, 0.0)
    ev = np.sort(np.linalg.eigvals(G.dense_from_csr(A)).real)
    lam = G._sum_spectrum([G.convdiff_1d_eigs(N, 50.0 / (N + 1)) for N in dims])
    np.testing.assert_allclose(ev, lam, atol=1e-9)


@pytest.mark.parametrize("dims,K", [((5, 4), 3), ((4, 3, 3), 5), ((6, 6), 4)])
def test_sigma_rule_gives_exact_count(dims, K):
    sig, k = G.sigma_for_negative_count([G.laplacian_1d_eigs(d) for d in dims], K)
    A = G.shifted_laplacian(dims, sig)
    ev = np.linalg.eigvalsh(G.dense_from_csr(A))
    assert k >= K and int((ev < 0).sum()) == k


def test_workload_sizes():
    w = C.lap2d_32_2x2_exact()
    assert w["A"].n == 1024 and w["nneg"] == 4
    w = C.lap3d_64_4x4x2_ilu0()
    assert w["A"].n == 262144 and w["A"].nnz == 1810432 and w["nneg"] == 20


def test_variable_kappa_symmetric_and_values_on_pattern():
    dims = (4, 3, 3)
    kap = G.kappa_field(dims, 0.5, 0)
    A = G.variable_kappa(dims, kap, 0.1)
    D = G.dense_from_csr(A)
    np.testing.assert_allclose(D, D.T, atol=0)
    # interior faces cancel in a row sum: what is left is kappa_i per boundary face, minus sigma
    _, _, _, _, nbnd = G._kappa_faces(dims)
    np.testing.assert_allclose(D.sum(1), nbnd * kap - 0.1, atol=1e-13)
    v = G.variable_kappa_values(dims, A, kap, 0.1)
    np.testing.assert_allclose(v, A.val, rtol=1e-15, atol=1e-15)


def test_variable_kappa_unit_kappa_is_laplacian():
    dims = (4, 3, 3)
    A1 = G.variable_kappa(dims, np.ones(36), 0.3)
    A2 = G.shifted_laplacian(dims, 0.3)
    np.testing.assert_array_equal(A1.rowptr, A2.rowptr)
    np.testing.assert_allclose(A1.val, A2.val, atol=1e-15)


def test_rhs_is_A_times_uniform():
    A = G.shifted_laplacian((5, 4), 0.1)
    b, xs = G.uniform_rhs(A, 0)
    assert xs.min() >= -1 and xs.max() <= 1
    np.testing.assert_allclose(b, G.dense_from_csr(A) @ xs, atol=1e-14)


def test_random_geometric_workload():
    """The matrix without a grid: symmetric, every diagonal stored, rows are
    neighbour counts (+1 near the boundary) minus the shift, and the shift of
    the 20,000-point workload leaves exactly one negative eigenvalue (shift-
    invert Lanczos for the smallest eigenvalues)."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    import scipy.sparse as sp

    w = C.rgg2d_20k()
    A = w["A"]
    M = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    assert abs(M - M.T).max() == 0
    d = M.diagonal()
    off = np.asarray((M != 0).sum(axis=1)).ravel() - 1
    assert np.all(np.isin(np.round(d + w["sigma"] - off, 12), (0.0, 1.0)))
    assert 10.0 < off.mean() < 14.0
    ev = np.sort(sla.eigsh(M, k=4, sigma=-0.01, which="LM", return_eigenvectors=False))
    assert (ev < 0).sum() == w["nneg"] == 1
