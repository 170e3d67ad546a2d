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
