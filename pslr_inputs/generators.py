"""Seeded synthetic test problems shaped like the paper's experiments (Section 4).

This module only builds inputs: sparse matrices in CSR form, right-hand sides and
seeded parameters.  It holds none of the PSLR method's arithmetic (no partition,
factorization, Schur complement, series or low-rank step), so both the FP64
oracle and the CUDA path can take their inputs from here.

Problems (all on the unit cube / square with zero Dirichlet boundary, 5- or
7-point stencils, lexicographic ordering ``idx = i + Nx*(j + Ny*k)``, x fastest):

* ``shifted_laplacian`` - Test 1 of Section 4, ``-Lap u - beta u``.  The stencil is
  the *unscaled* one (diagonal ``2d``, neighbours ``-1``) with ``sigma`` subtracted
  from the diagonal.  With this reading the closed-form spectrum reproduces the
  negative-eigenvalue counts printed in Section 4.1 (20/69/133 for 32^3/64^3/128^3
  at shifts .16/.08/.03, and 78 for 50^3 at shift .14).
* ``convection_diffusion`` - a Test-2-like nonsymmetric operator
  ``-Lap u + w.grad u - sigma u`` with ``w = Pe*(1,1,1)`` and first-order upwinding.
* ``variable_kappa`` - ``-div(kappa grad u) - sigma u`` with ``kappa = exp(g)``, g an
  i.i.d. seeded Gaussian per node; face coefficients are arithmetic means.

* ``random_geometric_laplacian`` - a matrix with no grid: the graph Laplacian of
  seeded random points in the unit square joined within a radius (mean degree
  about ``degree``), plus 1 on the diagonal of points within that radius of the
  boundary (as a Dirichlet neighbour would add), minus ``sigma``.  It stands in
  for the unstructured matrices of Section 4's Test 3, which are not available.

``sigma_for_negative_count`` turns "exactly / about K negative eigenvalues" into a
shift: it sorts the closed-form eigenvalues and puts sigma midway in the first gap
at or after the K-th eigenvalue.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR",
    "laplacian_1d_eigs",
    "convdiff_1d_eigs",
    "sigma_for_negative_count",
    "shifted_laplacian",
    "convection_diffusion",
    "variable_kappa",
    "kappa_field",
    "variable_kappa_values",
    "random_geometric_laplacian",
    "uniform_rhs",
    "csr_matvec",
    "dense_from_csr",
]


class CSR:
    """A square CSR matrix: int32 ``rowptr``/``col`` and float64 ``val``.

    Columns are sorted ascending inside every row and every diagonal entry is
    stored (the generators always emit it).
    """

    def __init__(self, n, rowptr, col, val, dims=None):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.dims = tuple(dims) if dims is not None else None

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def transpose(self):
        n = self.n
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(self.rowptr))
        order = np.lexsort((rows, self.col))
        col_t = rows[order].astype(np.int32)
        val_t = self.val[order]
        counts = np.bincount(self.col, minlength=n)
        rowptr_t = np.zeros(n + 1, dtype=np.int32)
        np.cumsum(counts, out=rowptr_t[1:])
        return CSR(n, rowptr_t, col_t, val_t, self.dims)


def _assemble(n, rows, cols, vals, dims):
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    vals = vals[order].astype(np.float64)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr, cols, vals, dims)


def _grid(dims):
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx
    for d in dims:
        coords.append(rem % d)
        rem = rem // d
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    return n, idx, coords, strides


def laplacian_1d_eigs(N):
    """Eigenvalues of tridiag(-1, 2, -1) of order N: 4 sin^2(pi k / (2(N+1)))."""
    k = np.arange(1, N + 1, dtype=np.float64)
    return 4.0 * np.sin(np.pi * k / (2.0 * (N + 1))) ** 2


def convdiff_1d_eigs(N, a):
    """Eigenvalues of tridiag(-1-a, 2+a, -1): 2 + a - 2 sqrt(1+a) cos(pi k/(N+1))."""
    k = np.arange(1, N + 1, dtype=np.float64)
    return 2.0 + a - 2.0 * np.sqrt(1.0 + a) * np.cos(np.pi * k / (N + 1))


def _sum_spectrum(eig1d_list):
    """All sums lambda_1[k1] + lambda_2[k2] + ... (the separable spectrum), sorted."""
    tot = np.zeros(1)
    for e in eig1d_list:
        tot = (tot[:, None] + e[None, :]).ravel()
    return np.sort(tot)


def sigma_for_negative_count(eig1d_list, K):
    """Shift sigma so that ``spectrum - sigma`` has exactly k >= K negative values.

    k is the smallest count >= K that falls in a gap of the sorted spectrum
    (lambda_k < lambda_{k+1}); sigma is the midpoint of that gap.  Returns
    ``(sigma, k)``.
    """
    lam = _sum_spectrum(eig1d_list)
    k = int(K)
    while k < lam.size and not (lam[k - 1] < lam[k]):
        k += 1
    if k >= lam.size:
        raise ValueError("no spectral gap at or after K")
    return 0.5 * (lam[k - 1] + lam[k]), k


def shifted_laplacian(dims, sigma):
    """Unscaled (2d)-point Laplacian minus sigma*I on a len(dims)-D grid."""
    n, idx, coords, strides = _grid(dims)
    nd = len(dims)
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 2.0 * nd - sigma)]
    for d in range(nd):
        for sgn in (-1, 1):
            c = coords[d] + sgn
            m = (c >= 0) & (c < dims[d])
            rows.append(idx[m])
            cols.append(idx[m] + sgn * strides[d])
            vals.append(np.full(int(m.sum()), -1.0))
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), dims)


def convection_diffusion(dims, peclet, sigma):
    """Upwinded -Lap u + w.grad u - sigma u, w = Pe*(1,..,1), scaled by h^2.

    Direction d has h_d = 1/(N_d+1) and a_d = Pe*h_d; its 1D operator is
    tridiag(-1-a_d, 2+a_d, -1) (upwind neighbour on the minus side), and the
    matrix is the sum of the 1D operators over the directions minus sigma*I.
    On a cube (one h) this is the h^2-scaled upwind discretisation.
    """
    n, idx, coords, strides = _grid(dims)
    nd = len(dims)
    a = [peclet / (N + 1.0) for N in dims]
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 2.0 * nd + sum(a) - sigma)]
    for d in range(nd):
        for sgn, w in ((-1, -1.0 - a[d]), (1, -1.0)):
            c = coords[d] + sgn
            m = (c >= 0) & (c < dims[d])
            rows.append(idx[m])
            cols.append(idx[m] + sgn * strides[d])
            vals.append(np.full(int(m.sum()), w))
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), dims)


def kappa_field(dims, std=0.5, seed=0):
    """kappa = exp(g), g ~ N(0, std^2) i.i.d. per node (numpy PCG64, ``seed``)."""
    n = int(np.prod(dims))
    g = np.random.default_rng(seed).normal(0.0, std, n)
    return np.exp(g)


def _kappa_faces(dims):
    """Face list of the 2d-point stencil: (row, col, dir) for in-grid neighbours,
    and (row, boundary-face count) for Dirichlet faces."""
    n, idx, coords, strides = _grid(dims)
    rows, cols = [], []
    nbnd = np.zeros(n, dtype=np.int64)
    for d in range(len(dims)):
        for sgn in (-1, 1):
            c = coords[d] + sgn
            m = (c >= 0) & (c < dims[d])
            rows.append(idx[m])
            cols.append(idx[m] + sgn * strides[d])
            nbnd += (~m).astype(np.int64)
    return n, idx, np.concatenate(rows), np.concatenate(cols), nbnd


def variable_kappa(dims, kappa, sigma):
    """-div(kappa grad u) - sigma u, 2d-point stencil, Dirichlet boundary.

    Interior face (i,j): coefficient (kappa_i + kappa_j)/2 on both rows.  A face
    on the boundary uses kappa_i.  Diagonal = sum of the row's face
    coefficients - sigma; off-diagonal (i,j) = -(face coefficient).
    """
    n, idx, r, c, nbnd = _kappa_faces(dims)
    kappa = np.asarray(kappa, dtype=np.float64)
    face = 0.5 * (kappa[r] + kappa[c])
    diag = np.bincount(r, weights=face, minlength=n) + nbnd * kappa - sigma
    rows = np.concatenate([idx, r])
    cols = np.concatenate([idx, c])
    vals = np.concatenate([diag, -face])
    return _assemble(n, rows, cols, vals, dims)


def variable_kappa_values(dims, A, kappa, sigma, xp=np):
    """Values of ``variable_kappa(dims, kappa, sigma)`` on A's CSR pattern.

    Written with plain array operations so that ``xp`` may be ``torch`` and the
    values stay differentiable in kappa (the chain rule from dL/dA_ij to
    dL/dkappa).  A must be the matrix ``variable_kappa`` returned for these dims.
    """
    n = A.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.rowptr))
    cols = A.col.astype(np.int64)
    _, _, _, _, nbnd = _kappa_faces(dims)
    off = rows != cols
    if xp is np:
        kr, kc = kappa[rows], kappa[cols]
        face = 0.5 * (kr + kc)
        diag = np.bincount(rows[off], weights=face[off], minlength=n) + nbnd * kappa - sigma
        out = np.where(off, -face, diag[rows])
        return out
    import torch  # plumbing only: keeps kappa -> A(kappa) differentiable

    rows_t = torch.as_tensor(rows, device=kappa.device)
    cols_t = torch.as_tensor(cols, device=kappa.device)
    off_t = torch.as_tensor(off, device=kappa.device)
    nb = torch.as_tensor(nbnd, dtype=kappa.dtype, device=kappa.device)
    face = 0.5 * (kappa[rows_t] + kappa[cols_t])
    diag = torch.zeros(n, dtype=kappa.dtype, device=kappa.device)
    diag = diag.index_add(0, rows_t[off_t], face[off_t]) + nb * kappa - sigma
    return torch.where(off_t, -face, diag[rows_t])


def random_geometric_laplacian(n, degree=8.0, sigma=0.05, seed=0):
    """Graph Laplacian of n seeded uniform points in [0,1]^2, pairs closer than
    r = sqrt(degree / (pi n)) joined with weight -1, the diagonal holding the
    number of neighbours, +1 for points within r of the boundary, - sigma.
    Rows in the order the points were drawn (no spatial ordering)."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = float(np.sqrt(degree / (np.pi * n)))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray").astype(np.int64)
    i, j = pairs[:, 0], pairs[:, 1]
    deg = np.bincount(i, minlength=n) + np.bincount(j, minlength=n)
    near = ((pts < r) | (pts > 1.0 - r)).any(axis=1)
    diag = deg + near.astype(np.float64) - sigma
    rows = np.concatenate([i, j, np.arange(n)])
    cols = np.concatenate([j, i, np.arange(n)])
    vals = np.concatenate([-np.ones(2 * len(i)), diag])
    return _assemble(n, rows, cols, vals, None)


def uniform_rhs(A, seed=0, nrhs=1):
    """x* ~ U[-1,1] (numpy PCG64, ``seed``) and b = A x*.  Shapes (n,) or (n, nrhs),
    column-major when nrhs > 1 (each column is contiguous in the returned
    Fortran-ordered arrays)."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        xs = rng.uniform(-1.0, 1.0, A.n)
        return csr_matvec(A, xs), xs
    xs = np.asfortranarray(rng.uniform(-1.0, 1.0, (nrhs, A.n)).T)
    b = np.asfortranarray(np.stack([csr_matvec(A, xs[:, j]) for j in range(nrhs)], axis=1))
    return b, xs


def csr_matvec(A, x):
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr))
    return np.bincount(rows, weights=A.val * x[A.col], minlength=A.n)


def dense_from_csr(A):
    D = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr))
    D[rows, A.col] = A.val
    return D
