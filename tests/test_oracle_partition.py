"""Pins for the oracle's graph partition (recursive bisection of breadth-first
level structures from George-Liu pseudo-peripheral vertices), which stands in
for the paper's METIS partition (Section 2) on matrices without a grid."""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import generators as G


def _csr_from_edges(n, edges, diag=4.0):
    rows = [i for i in range(n)] + [a for a, b in edges] + [b for a, b in edges]
    cols = [i for i in range(n)] + [b for a, b in edges] + [a for a, b in edges]
    vals = [diag] * n + [-1.0] * (2 * len(edges))
    return G._assemble(n, np.array(rows), np.array(cols), np.array(vals, dtype=float), None)


def _sizes(n, k):
    """Part sizes the recursive split must produce: floor(n (k//2) / k) to
    the first k//2 parts, the rest to the others."""
    if k == 1:
        return [n]
    k1 = k // 2
    n1 = n * k1 // k
    return _sizes(n1, k1) + _sizes(n - n1, k - k1)


@pytest.mark.parametrize("n,k", [(37, 1), (37, 2), (37, 5), (64, 8), (100, 7)])
def test_shuffled_path_is_cut_into_consecutive_runs(n, k):
    """On a path graph (vertices relabelled at random) breadth-first order runs
    from one end to the other, so every part is a run of consecutive path
    positions and the runs have the sizes of the recursive split."""
    lab = np.random.default_rng(n + k).permutation(n)  # path position t carries label lab[t]
    A = _csr_from_edges(n, [(lab[t], lab[t + 1]) for t in range(n - 1)])
    part = O.graph_partition(A, k)
    along = part[lab]
    runs = [along[0]]
    for p in along[1:]:
        if p != runs[-1]:
            runs.append(p)
    assert len(runs) == k and len(set(runs)) == k  # each part one run
    counts = np.bincount(part, minlength=k)
    assert sorted(counts.tolist()) == sorted(_sizes(n, k))


def test_grid_bisection_follows_the_corner_levels():
    """8x8 grid, 2 parts: vertex 0 is a corner, the search from it ends at the
    opposite corner with the same number of levels, so the order runs along
    anti-diagonals from vertex 0.  The first 32 vertices are the 28 with
    i + j <= 6 and 4 of the 8 with i + j = 7."""
    A = G.shifted_laplacian((8, 8), 0.0)
    part = O.graph_partition(A, 2)
    i, j = np.arange(64) % 8, np.arange(64) // 8
    p0 = part[0]
    assert np.all(part[i + j <= 6] == p0)
    assert np.sum(part[i + j == 7] == p0) == 4
    assert np.all(part[i + j >= 8] != p0)
    assert np.sum(part == p0) == 32


def test_components_are_listed_by_smallest_vertex():
    """Two disjoint paths, the one holding vertex 0 listed first: with 2 parts
    and equal halves the first part is exactly that path."""
    n = 20
    even = [(a, a + 2) for a in range(0, n - 2, 2)]  # path over even labels
    odd = [(a, a + 2) for a in range(1, n - 2, 2)]   # path over odd labels
    A = _csr_from_edges(n, even + odd)
    part = O.graph_partition(A, 2)
    assert np.all(part[0::2] == part[0]) and np.all(part[1::2] != part[0])


def test_every_vertex_once_and_sizes_on_a_random_graph():
    A = G.random_geometric_laplacian(3000, 10.0, 0.0, 1)
    for k in (3, 16, 33):
        part = O.graph_partition(A, k)
        assert part.min() == 0 and part.max() == k - 1
        assert sorted(np.bincount(part, minlength=k).tolist()) == sorted(_sizes(A.n, k))


def test_argument_errors():
    A = G.shifted_laplacian((4, 4), 0.0)
    for k in (0, 17):
        with pytest.raises(O.OracleError):
            O.graph_partition(A, k)
