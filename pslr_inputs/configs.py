"""Named synthetic workloads (the paper's Section-4 problem families at GB300 sizes).

Every workload is a dict with the PSLR parameters (subdomain split, local
factor kind, series order m, rank r) and a ``build()`` that returns the matrix
and right-hand side(s).  Seeds: 0 for right-hand sides, kappa fields and the
batch's random sizes; 1 for the differentiable problem's target field.

Workloads (names say what they are):

``lap2d_32_2x2_exact``    2D 5-pt Laplacian 32x32, sigma for exactly 4 negative
                          eigenvalues, 2x2 split, exact dense local LU, m=3, r=8.
``lap3d_64_4x4x2_ilu0``   3D 7-pt Laplacian 64^3, sigma for 20 negative
                          eigenvalues, 4x4x2 split, ILU(0), m=3, r=16.
``batch2d_64sys``         64 shifted 2D Laplacians, side ~ U{64..256}, 4 rhs each.
``kappa3d_48_3x3x3``      3D 48^3 variable-kappa operator, 3x3x3 split, m=3, r=16.
``cd3d_128_8x8x4_ilu0``   3D 128^3 upwinded convection-diffusion, Pe=50, sigma for
                          20 negative eigenvalues of the shifted operator, 8x8x4
                          split, ILU(0), m=5, r=32.
``cd3d_128_8x8x4_ilu0_noshift``  the same operator without the shift (definite).
``lap3d_50_shift014``     3D 7-pt Laplacian 50^3 shifted by 0.14 (78 negative
                          eigenvalues: the strongly indefinite case of Section
                          4.1's rank study), 3x3x4 split (36 subdomains, near the
                          paper's s = 35), ILUT(1e-2) as in that study, m=3; the
                          rank is the variable.
``rgg2d_20k``             a matrix with no grid: the anchored graph Laplacian of
                          20,000 random points in the unit square (mean degree
                          12) shifted by 0.0064, between its two smallest
                          eigenvalues (one negative eigenvalue); 16 parts from
                          the graph partition, ILU(0), m=3, r=8.
"""
from __future__ import annotations

import numpy as np

from . import generators as G

FACTOR_ILU0 = 0
FACTOR_EXACT_LU = 1
FACTOR_ILUT = 2  # threshold ILU, drop tolerance ``drop_tol`` (Section 4 uses 1e-2)


def _lap(dims, K):
    sig, k = G.sigma_for_negative_count([G.laplacian_1d_eigs(d) for d in dims], K)
    return G.shifted_laplacian(dims, sig), sig, k


def lap2d_32_2x2_exact():
    A, sig, k = _lap((32, 32), 4)
    return dict(name="lap2d_32_2x2_exact", A=A, sigma=sig, nneg=k, ndim=2, dims=(32, 32, 1),
                splits=(2, 2, 1), factor=FACTOR_EXACT_LU, m=3, rank=8)


def lap3d_64_4x4x2_ilu0():
    A, sig, k = _lap((64, 64, 64), 20)
    return dict(name="lap3d_64_4x4x2_ilu0", A=A, sigma=sig, nneg=k, ndim=3, dims=(64, 64, 64),
                splits=(4, 4, 2), factor=FACTOR_ILU0, m=3, rank=16)


def cd3d_128_8x8x4_ilu0(N=128, splits=(8, 8, 4), m=5, rank=32, K=20):
    pe = 50.0
    a = pe / (N + 1.0)
    if K == 0:
        sig, k = 0.0, 0
    else:
        sig, k = G.sigma_for_negative_count([G.convdiff_1d_eigs(N, a)] * 3, K)
    A = G.convection_diffusion((N, N, N), pe, sig)
    name = f"cd3d_{N}_{splits[0]}x{splits[1]}x{splits[2]}_ilu0" + ("_noshift" if K == 0 else "")
    return dict(name=name, A=A, sigma=sig, nneg=k, ndim=3, dims=(N, N, N), splits=tuple(splits), factor=FACTOR_ILU0,
                m=m, rank=rank)


def cd3d_128_8x8x4_ilu0_noshift():
    """The same upwinded operator without the shift (definite, nonsymmetric):
    the 128^3 system on which restarted FGMRES reaches 1e-8."""
    return cd3d_128_8x8x4_ilu0(K=0)


def kappa3d_48_3x3x3(N=48, splits=(3, 3, 3), m=3, rank=16, K=10):
    dims = (N, N, N)
    sig, k = G.sigma_for_negative_count([G.laplacian_1d_eigs(N)] * 3, K)
    kap = G.kappa_field(dims, 0.5, seed=0)
    A = G.variable_kappa(dims, kap, sig)
    return dict(name=f"kappa3d_{N}_{splits[0]}x{splits[1]}x{splits[2]}", A=A, sigma=sig, nneg=k,
                ndim=3, dims=dims, splits=tuple(splits), factor=FACTOR_ILU0, m=m, rank=rank,
                kappa=kap)


def lap3d_50_shift014(rank=15, factor=FACTOR_ILUT, drop_tol=1e-2):
    dims = (50, 50, 50)
    sig = 0.14
    lam = G._sum_spectrum([G.laplacian_1d_eigs(d) for d in dims])
    A = G.shifted_laplacian(dims, sig)
    return dict(name="lap3d_50_shift014", A=A, sigma=sig, nneg=int((lam < sig).sum()), ndim=3, dims=dims,
                splits=(3, 3, 4), factor=factor, m=3, rank=rank, drop_tol=drop_tol)


def rgg2d_20k(n=20000, nparts=16, factor=FACTOR_ILU0, m=3, rank=8, drop_tol=1e-2):
    sig = 0.0064
    A = G.random_geometric_laplacian(n, 12.0, sig, 0)
    return dict(name="rgg2d_20k", A=A, sigma=sig, nneg=1, ndim=2, nparts=nparts, factor=factor, m=m, rank=rank,
                drop_tol=drop_tol)


def batch2d_64sys(nsys=64, lo=64, hi=256, nrhs=4, seed=0):
    """The batched workload: per system side N ~ U{lo..hi}, split ceil(N/32) per
    side clipped to [4, 8], m ~ U{2..5}, r ~ {8, 16, 32}, sigma for 4 negative
    eigenvalues, ILU(0)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, nsys)
    ms = rng.integers(2, 6, nsys)
    ranks = rng.choice(np.array([8, 16, 32]), nsys)
    systems = []
    for N, m, r in zip(sides.tolist(), ms.tolist(), ranks.tolist()):
        sp = int(min(8, max(4, -(-N // 32))))
        A, sig, k = _lap((N, N), 4)
        systems.append(dict(A=A, sigma=sig, nneg=k, ndim=2, dims=(N, N, 1), splits=(sp, sp, 1),
                            factor=FACTOR_ILU0, m=int(m), rank=int(r)))
    return dict(name=f"batch2d_{nsys}sys", systems=systems, nrhs=nrhs)


WORKLOADS = {
    "lap2d_32_2x2_exact": lap2d_32_2x2_exact,
    "lap3d_64_4x4x2_ilu0": lap3d_64_4x4x2_ilu0,
    "batch2d_64sys": batch2d_64sys,
    "kappa3d_48_3x3x3": kappa3d_48_3x3x3,
    "cd3d_128_8x8x4_ilu0": cd3d_128_8x8x4_ilu0,
    "cd3d_128_8x8x4_ilu0_noshift": cd3d_128_8x8x4_ilu0_noshift,
    "lap3d_50_shift014": lap3d_50_shift014,
    "rgg2d_20k": rgg2d_20k,
}


def small_problem(kind, dims, splits, factor=FACTOR_ILU0, m=3, rank=4, K=2, seed=0, drop_tol=1e-2):
    """A small problem of any family, for tests that must span several tiles and
    ragged tails while the oracle finishes in seconds."""
    nd = len(dims)
    if kind == "lap":
        A, sig, k = _lap(dims, K)
    elif kind == "cd":
        sig, k = G.sigma_for_negative_count([G.convdiff_1d_eigs(N, 50.0 / (N + 1.0)) for N in dims], K)
        A = G.convection_diffusion(dims, 50.0, sig)
    elif kind == "kappa":
        sig, k = G.sigma_for_negative_count([G.laplacian_1d_eigs(d) for d in dims], K)
        A = G.variable_kappa(dims, G.kappa_field(dims, 0.5, seed), sig)
    else:
        raise ValueError(kind)
    d3 = tuple(dims) + (1,) * (3 - nd)
    s3 = tuple(splits) + (1,) * (3 - nd)
    return dict(name=f"{kind}{nd}d_{'x'.join(map(str, dims))}", A=A, sigma=sig, nneg=k, ndim=nd,
                dims=d3, splits=s3, factor=factor, m=m, rank=rank, drop_tol=drop_tol)
