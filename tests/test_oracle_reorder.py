"""Pins for the oracle's reordering and block extraction (Section 2, Eq. 2.1, Eq. 3.1)."""
import os

import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    d = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = np.array([int(x) for x in v], dtype=np.int32)
    return d


@pytest.mark.parametrize("fname", ["partition_grid4x4_split2x2.txt", "partition_chain9_split3.txt"])
def test_partition_golden(fname):
    g = _read_golden(fname)
    dims = tuple(int(x) for x in g["dims"] if x > 1) or (int(g["dims"][0]),)
    A = G.shifted_laplacian(dims, 0.0)
    o = O.Oracle(A, dims=g["dims"], splits=g["splits"], factor=0)
    part, iface, perm = o.maps()
    io, go = o.offsets()
    np.testing.assert_array_equal(part, g["part"])
    np.testing.assert_array_equal(iface, g["iface"])
    np.testing.assert_array_equal(perm, g["perm"])
    np.testing.assert_array_equal(io, g["interior_off"])
    np.testing.assert_array_equal(go, g["interface_off"])


CASES = [
    ("lap", (12, 10), (3, 2)),
    ("lap", (6, 5, 4), (2, 2, 2)),
    ("cd", (6, 6, 6), (3, 2, 1)),
    ("kappa", (5, 6, 4), (2, 3, 1)),
]


@pytest.mark.parametrize("kind,dims,splits", CASES)
def test_reordering_invariants(kind, dims, splits):
    w = C.small_problem(kind, dims, splits)
    A = w["A"]
    o = O.from_workload(w)
    part, iface, perm = o.maps()
    n = A.n
    # perm is a permutation; interiors first
    assert sorted(perm.tolist()) == list(range(n))
    assert o.p == int((iface == 0).sum()) and o.q == n - o.p
    assert np.all(iface[perm[: o.p]] == 0) and np.all(iface[perm[o.p:]] == 1)
    # edge separator: interior nodes only couple inside their part,
    # every interface node couples to another part (pattern of A + A^T)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    cross = (part[rows] != part[A.col]) & (rows != A.col)
    touched = np.zeros(n, bool)
    touched[rows[cross]] = True
    touched[A.col[cross]] = True
    np.testing.assert_array_equal(touched, iface.astype(bool))
    # subdomain order, original order inside a subdomain
    io, go = o.offsets()
    for i in range(o.s):
        blk = perm[io[i]:io[i + 1]]
        assert np.all(part[blk] == i) and np.all(np.diff(blk) > 0)
        blk = perm[o.p + go[i]:o.p + go[i + 1]]
        assert np.all(part[blk] == i) and np.all(np.diff(blk) > 0)


@pytest.mark.parametrize("kind,dims,splits", CASES)
def test_blocks_reassemble_and_are_block_diagonal(kind, dims, splits):
    w = C.small_problem(kind, dims, splits)
    A = w["A"]
    o = O.from_workload(w)
    part, iface, perm = o.maps()
    D = G.dense_from_csr(A)
    PA = D[np.ix_(perm, perm)]
    p = o.p
    B, E, F, Cc = (o.dense_block(x) for x in ("B", "E", "F", "C"))
    np.testing.assert_array_equal(np.block([[B, E], [F, Cc]]), PA)
    C0, Cg = o.dense_block("C0"), o.dense_block("Cg")
    np.testing.assert_array_equal(C0 + Cg, Cc)
    io, go = o.offsets()
    pi = np.repeat(np.arange(o.s), np.diff(io))  # part of each interior row
    pg = np.repeat(np.arange(o.s), np.diff(go))  # part of each interface row
    # B, E, F and C0 are block diagonal by subdomain (Section 2); C_g has no
    # entry inside a subdomain (it is C stripped of its diagonal blocks).
    assert np.all(B[pi[:, None] != pi[None, :]] == 0)
    assert np.all(E[pi[:, None] != pg[None, :]] == 0)
    assert np.all(F[pg[:, None] != pi[None, :]] == 0)
    assert np.all(C0[pg[:, None] != pg[None, :]] == 0)
    assert np.all(Cg[pg[:, None] == pg[None, :]] == 0)
    # F has the block structure of E^T
    np.testing.assert_array_equal(F != 0, (E != 0).T)


def test_single_subdomain_has_no_interface():
    A = G.shifted_laplacian((6, 5), 0.2)
    o = O.Oracle(A, dims=(6, 5, 1), splits=(1, 1, 1))
    assert o.q == 0 and o.p == 30
    _, _, perm = o.maps()
    np.testing.assert_array_equal(perm, np.arange(30))
