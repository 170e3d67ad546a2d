"""Pins for the oracle's local factors (Algorithm 1, steps 2-5) and their solves."""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

from conftest import dense_lu_product


@pytest.mark.parametrize("kind,dims,splits", [
    ("lap", (12, 10), (3, 2)), ("cd", (6, 6, 6), (3, 2, 1)), ("kappa", (5, 6, 4), (2, 3, 1))])
def test_ilu0_matches_A_on_its_pattern(kind, dims, splits):
    """ILU(0) is characterised by (L U)_ij = a_ij for every (i,j) in the pattern
    of the factored matrix (Saad, Iterative Methods, Sec. 10.3.2)."""
    o = O.from_workload(C.small_problem(kind, dims, splits))
    for blk, fac in (("B", "LU_B"), ("C0", "LU_C0")):
        M = o.dense_block(blk)
        LU = dense_lu_product(o, fac)
        pat = o.dense_block(fac) != 0
        pat |= M != 0
        np.testing.assert_allclose(LU[M != 0], M[M != 0], rtol=1e-13, atol=1e-13)
        # and the factor has exactly the pattern of the block
        np.testing.assert_array_equal(o.dense_block(fac) != 0, M != 0)


def test_ilu0_on_tridiagonal_blocks_is_exact():
    """A 1D chain has tridiagonal blocks, whose LU has no fill: ILU(0) = LU and
    B~^{-1} must equal LAPACK's solve."""
    A = G.shifted_laplacian((40,), 0.3)
    o = O.Oracle(A, dims=(40, 1, 1), splits=(4, 1, 1), factor=0)
    B = o.dense_block("B")
    v = np.random.default_rng(0).uniform(-1, 1, o.p)
    np.testing.assert_allclose(o.solve_B(v), np.linalg.solve(B, v), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(o.solve_BT(v), np.linalg.solve(B.T, v), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dims,splits", [((12, 10), (3, 2)), ((32, 32), (2, 2))])
def test_exact_lu_solves_equal_lapack(dims, splits):
    w = C.small_problem("lap", dims, splits, factor=1, K=4)
    o = O.from_workload(w)
    rng = np.random.default_rng(1)
    for blk, solve, solve_t, n in (("B", o.solve_B, o.solve_BT, o.p), ("C0", o.solve_C0, o.solve_C0T, o.q)):
        M = o.dense_block(blk)
        v = rng.uniform(-1, 1, n)
        ref = np.linalg.solve(M, v)
        np.testing.assert_allclose(solve(v), ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
        ref = np.linalg.solve(M.T, v)
        np.testing.assert_allclose(solve_t(v), ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_ilu_solves_invert_LU_product():
    o = O.from_workload(C.small_problem("cd", (6, 6, 6), (3, 2, 1)))
    rng = np.random.default_rng(2)
    for fac, solve, solve_t, n in (("LU_B", o.solve_B, o.solve_BT, o.p),
                                   ("LU_C0", o.solve_C0, o.solve_C0T, o.q)):
        M = dense_lu_product(o, fac)
        v = rng.uniform(-1, 1, n)
        np.testing.assert_allclose(M @ solve(v), v, atol=1e-12)
        np.testing.assert_allclose(M.T @ solve_t(v), v, atol=1e-12)


def test_zero_pivot_is_reported():
    A = G.shifted_laplacian((6, 5), 0.0)
    A.val[A.rowptr[0]] = 0.0  # a_00 = 0: the first pivot of B_1 vanishes
    with pytest.raises(O.OracleError) as e:
        O.Oracle(A, dims=(6, 5, 1), splits=(2, 1, 1), factor=0)
    assert e.value.status == O.ERR_ZERO_PIVOT


# ---------------------------------------------------------------- ILUT(tau)

def _row_scales(M):
    """Mean modulus of the stored entries of each row (SPARSKIT's ilut
    scale): computed here from the dense block, independently of the oracle."""
    return np.abs(M).sum(axis=1) / np.count_nonzero(M, axis=1)


def test_ilut_without_dropping_is_exact_lu():
    """tau = 0 drops nothing: ILUT is the complete LU without pivoting, so
    L U = B exactly and the solves equal LAPACK's (an SPD shifted Laplacian,
    where LU without pivoting exists)."""
    A = G.shifted_laplacian((7, 6, 5), -0.5)
    o = O.Oracle(A, dims=(7, 6, 5), splits=(2, 2, 1), factor=2, drop_tol=0.0)
    for blk, fac, solve, n in (("B", "LU_B", o.solve_B, o.p), ("C0", "LU_C0", o.solve_C0, o.q)):
        M = o.dense_block(blk)
        np.testing.assert_allclose(dense_lu_product(o, fac), M, atol=1e-12 * np.abs(M).max())
        v = np.random.default_rng(3).uniform(-1, 1, n)
        np.testing.assert_allclose(solve(v), np.linalg.solve(M, v), rtol=1e-10, atol=1e-12)


def test_ilut_on_tridiagonal_blocks_equals_ilu0():
    """A 1D chain's blocks are tridiagonal: their LU has no fill and every
    multiplier is far above 1e-2 of the row's mean modulus, so ILUT(1e-2) =
    ILU(0)."""
    A = G.shifted_laplacian((40,), 0.3)
    o0 = O.Oracle(A, dims=(40, 1, 1), splits=(4, 1, 1), factor=0)
    ot = O.Oracle(A, dims=(40, 1, 1), splits=(4, 1, 1), factor=2, drop_tol=1e-2)
    for fac in ("LU_B", "LU_C0"):
        a, b = o0.dense_block(fac), ot.dense_block(fac)
        np.testing.assert_array_equal(a != 0, b != 0)
        np.testing.assert_allclose(b, a, rtol=1e-14, atol=0)


def test_ilut_huge_tolerance_keeps_only_the_diagonal():
    """With tau far above every ratio |a_ij| / mean|a_i|, every multiplier and
    every off-diagonal entry is dropped: L = 0 and U = diag(B)."""
    w = C.small_problem("cd", (6, 5, 4), (2, 2, 1), factor=2, drop_tol=10.0)
    o = O.from_workload(w)
    for blk, fac in (("B", "LU_B"), ("C0", "LU_C0")):
        F = o.dense_block(fac)
        np.testing.assert_array_equal(F, np.diag(np.diag(o.dense_block(blk))))


@pytest.mark.parametrize("kind,dims,splits", [("lap", (8, 7, 6), (2, 2, 1)), ("cd", (7, 6, 5), (2, 2, 2))])
def test_ilut_keeps_only_entries_above_the_threshold(kind, dims, splits):
    """Every stored off-diagonal entry of the factors is at least
    tau mean|a_i| in modulus (mean modulus of the block row), every diagonal is
    stored, and the fill lies between ILU(0)'s and the exact LU's."""
    tau = 1e-2
    w = C.small_problem(kind, dims, splits, factor=2, drop_tol=tau)
    o = O.from_workload(w)
    o0 = O.from_workload(dict(w, factor=0))
    for blk, fac in (("B", "LU_B"), ("C0", "LU_C0")):
        M, F = o.dense_block(blk), o.dense_block(fac)
        tol = tau * _row_scales(M)
        off = F.copy()
        np.fill_diagonal(off, 0.0)
        rows, cols = np.nonzero(off)
        assert np.all(np.abs(off[rows, cols]) >= tol[rows])
        assert np.all(np.diag(F) != 0)
        nnz_t, nnz_0 = np.count_nonzero(F), np.count_nonzero(o0.dense_block(fac))
        assert nnz_t >= nnz_0 * 0.5 and nnz_t <= F.shape[0] ** 2


def test_ilut_matches_its_definition_on_a_tiny_block():
    """Brute force: ILUT(tau) row by row on dense rows, as the definition
    reads, on a tiny convection-diffusion block; the oracle's sparse version
    must store exactly these values."""
    tau = 0.05
    w = C.small_problem("cd", (4, 3, 3), (2, 1, 1), factor=2, drop_tol=tau)
    o = O.from_workload(w)
    M = o.dense_block("B")
    n = M.shape[0]
    LU = np.zeros((n, n))
    for i in range(n):
        wrow = M[i].copy()
        nzs = [abs(x) for x in M[i] if x != 0]
        tol = tau * (sum(nzs) / len(nzs))
        for k in range(i):
            if wrow[k] == 0.0:
                continue
            mult = wrow[k] / LU[k, k]
            if abs(mult) < tol:
                wrow[k] = 0.0
                continue
            wrow[k] = mult
            for j in range(k + 1, n):
                if LU[k, j] != 0.0:
                    wrow[j] -= mult * LU[k, j]
        for j in range(n):
            if j != i and abs(wrow[j]) < tol:
                wrow[j] = 0.0
        LU[i] = wrow
    np.testing.assert_allclose(o.dense_block("LU_B"), LU, rtol=1e-13, atol=1e-15)
