"""Pins for the low-rank step (Eq. 3.16-3.18, Algorithm 1), Algorithm 3, its
transpose and FGMRES."""
import os

import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

from conftest import dense_operators

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _columns(fn, q):
    return np.stack([fn(e) for e in np.eye(q)], axis=1)


def _ops(kind, dims, splits, factor, K=3):
    w = C.small_problem(kind, dims, splits, factor=factor, K=K)
    o = O.from_workload(w)
    D = dense_operators(o, factor)
    Es = -D["Cg"] + D["F"] @ np.linalg.solve(D["Bt"], D["E"])
    return w, o, D, Es


def test_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014), seed 0: the reference generator's
    first outputs, mapped to [-1, 1) by the top 53 bits."""
    vals = [int(l.split()[1], 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for j, z in enumerate(vals):
        assert O.splitmix_uniform(0, j) == (z >> 11) * 2.0 ** -53 * 2.0 - 1.0


@pytest.mark.parametrize("kind,dims,splits,factor,m,r", [
    ("lap", (12, 10), (3, 2), 1, 3, 6),
    ("cd", (6, 6, 6), (3, 2, 1), 0, 2, 8),
    ("kappa", (5, 6, 4), (2, 3, 1), 0, 3, 5),
])
def test_arnoldi_relations(kind, dims, splits, factor, m, r):
    """Eq. 3.16: V has orthonormal columns, H = V^T E_rr V is upper Hessenberg and
    E_rr v_j = sum_{i<=j+1} h_ij v_i for j < r (the Arnoldi relation)."""
    w, o, D, Es = _ops(kind, dims, splits, factor)
    Err = np.linalg.matrix_power(Es @ np.linalg.inv(D["C0t"]), m + 1)
    k, st = o.build_lowrank(m, r, seed=7)
    assert k == r and st == O.OK
    V, H, Gm = o.lowrank()
    np.testing.assert_allclose(V.T @ V, np.eye(r), atol=1e-12)
    sc = max(1.0, np.abs(Err).max())
    np.testing.assert_allclose(V.T @ Err @ V, H, atol=1e-10 * sc)
    assert np.all(np.abs(np.tril(H, -2)) <= 1e-10 * sc)
    np.testing.assert_allclose(Err @ V[:, :-1], V @ H[:, :-1], atol=1e-10 * sc)
    # start vector = normalised SplitMix64 draws
    u = np.array([O.splitmix_uniform(7, j) for j in range(o.q)])
    np.testing.assert_allclose(V[:, 0], u / np.linalg.norm(u), atol=1e-15)
    # Eq. 3.17 via Sherman-Morrison-Woodbury: (I - V H V^T)(I + V G V^T) = I
    q = o.q
    np.testing.assert_allclose((np.eye(q) - V @ H @ V.T) @ (np.eye(q) + V @ Gm @ V.T), np.eye(q),
                               atol=1e-10 * max(1.0, np.abs(Gm).max()))
    np.testing.assert_allclose(Gm, np.linalg.inv(np.eye(r) - H) - np.eye(r), atol=1e-10)


def test_arnoldi_frobenius_error_monotone_in_rank():
    """Sec. 3.2: ||E_rr(m) - V H V^T||_F decreases monotonically as r grows."""
    w, o, D, Es = _ops("lap", (12, 10), (3, 2), 1)
    m = 2
    Err = np.linalg.matrix_power(Es @ np.linalg.inv(D["C0t"]), m + 1)
    errs = []
    for r in range(1, 12):
        o.build_lowrank(m, r, seed=3)
        V, H, _ = o.lowrank()
        errs.append(np.linalg.norm(Err - V @ H @ V.T, "fro"))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))


def test_full_rank_eigenvalues_match_brute_force():
    w, o, D, Es = _ops("lap", (12, 10), (3, 2), 1)
    m = 1
    Err = np.linalg.matrix_power(Es @ np.linalg.inv(D["C0t"]), m + 1)
    k, st = o.build_lowrank(m, o.q, seed=0, full_rank=True)
    assert k == o.q
    V, H, _ = o.lowrank()
    ev_h = np.sort_complex(np.linalg.eigvals(H))
    ev_e = np.sort_complex(np.linalg.eigvals(Err))
    np.testing.assert_allclose(ev_h, ev_e, atol=1e-8)


def test_partial_rank_finds_the_outlier_and_lowers_iterations():
    """Sec. 4.1.3 on a small indefinite problem (16^3, 12 negative
    eigenvalues, 2x2x2, ILUT(1e-2), m = 3): E_rr(m), formed column by column
    here, has eigenvalues of modulus above 1; 20 Arnoldi steps find the
    largest of them (largest-modulus eigenvalue of H against the brute-force
    spectrum), and the low-rank term lowers the FGMRES(127) iteration count
    as r grows (0 -> 20 -> 40)."""
    dims = (16, 16, 16)
    lam = np.sort(G._sum_spectrum([G.laplacian_1d_eigs(d) for d in dims]))
    A = G.shifted_laplacian(dims, 0.5 * (lam[11] + lam[12]))
    o = O.Oracle(A, dims=dims, splits=(2, 2, 2), factor=2, drop_tol=1e-2)
    m, q = 3, o.q
    Err = np.column_stack([o.Err(m, e) for e in np.eye(q)])
    ev = np.linalg.eigvals(Err)
    top = np.abs(ev).max()
    assert top > 1.0
    b, _ = G.uniform_rhs(A, 0)
    its = []
    for r in (0, 20, 40):
        if r:
            k, st = o.build_lowrank(m, r, seed=0)
            assert k == r
            H = o.lowrank()[1]
            if r == 20:
                assert abs(np.abs(np.linalg.eigvals(H)).max() - top) <= 1e-6 * top
        else:
            o.set_lowrank(m, np.zeros((q, 0)), np.zeros((0, 0)))
        x, it, rel, st = o.fgmres(b, rtol=1e-8, restart=127, maxit=2000)
        assert st == O.OK
        its.append(it)
    assert its[0] > its[1] > its[2], its


def test_breakdown_truncates_rank():
    """On a 4x4 grid cut 2x2 the interface operator has the square's symmetry, so
    E_rr(m) has repeated eigenvalues and a Krylov space of dimension < q: Arnoldi
    breaks down (h_{j+1,j} ~ 0).  Truncated, V spans an invariant subspace, so
    E_rr V = V H holds with no remainder; in full-rank mode fresh directions
    complete V to the whole space."""
    A = G.shifted_laplacian((4, 4), 0.0)
    o = O.Oracle(A, dims=(4, 4, 1), splits=(2, 2, 1), factor=1)
    q = o.q
    k, st = o.build_lowrank(1, q, seed=0)
    assert st == O.ERR_BREAKDOWN and 0 < k < q
    V, H, _ = o.lowrank()
    Err = _columns(lambda v: o.Err(1, v), q)
    np.testing.assert_allclose(Err @ V, V @ H, atol=1e-12)
    k, st = o.build_lowrank(1, q, seed=0, full_rank=True)
    assert st == O.OK and k == q
    V, H, _ = o.lowrank()
    np.testing.assert_allclose(V.T @ V, np.eye(q), atol=1e-12)
    np.testing.assert_allclose(V.T @ Err @ V, H, atol=1e-12)
    k, st = o.build_lowrank(1, q + 5, seed=0, full_rank=True)
    assert k == q


def _dense_Minv(o, D, m, V, Gm):
    """Block form of Algorithm 3: M^{-1} = [[B^{-1} + B^{-1} E K F B^{-1}, -B^{-1} E K],
    [-K F B^{-1}, K]], K = P_m (I + V G V^T), P_m = sum_i (C0^{-1}E_s)^i C0^{-1}."""
    q = o.q
    Bi = np.linalg.inv(D["Bt"])
    C0i = np.linalg.inv(D["C0t"])
    Es = -D["Cg"] + D["F"] @ Bi @ D["E"]
    N = C0i @ Es
    Pm = sum(np.linalg.matrix_power(N, i) for i in range(m + 1)) @ C0i
    K = Pm @ (np.eye(q) + V @ Gm @ V.T)
    E, F = D["E"], D["F"]
    return np.block([[Bi + Bi @ E @ K @ F @ Bi, -Bi @ E @ K], [-K @ F @ Bi, K]])


@pytest.mark.parametrize("kind,dims,splits,factor,m,r", [
    ("lap", (12, 10), (3, 2), 1, 3, 6),
    ("lap", (12, 10), (3, 2), 0, 0, 0),
    ("cd", (6, 6, 6), (3, 2, 1), 0, 2, 8),
    ("kappa", (5, 6, 4), (2, 3, 1), 0, 3, 5),
    ("lap", (6, 5, 4), (2, 2, 2), 0, 5, 4),
])
def test_apply_equals_block_formula(kind, dims, splits, factor, m, r):
    w, o, D, Es = _ops(kind, dims, splits, factor)
    if r:
        o.build_lowrank(m, r, seed=1)
    else:
        o.set_lowrank(m, None, None)
    V, H, Gm = o.lowrank()
    Minv = _dense_Minv(o, D, m, V, Gm)
    _, _, perm = o.maps()
    Mo = np.empty_like(Minv)  # back to the original ordering
    Mo[np.ix_(perm, perm)] = Minv
    got = _columns(o.apply, o.n)
    sc = np.abs(Mo).max()
    np.testing.assert_allclose(got, Mo, atol=1e-11 * sc)
    gotT = _columns(o.apply_T, o.n)
    np.testing.assert_allclose(gotT, Mo.T, atol=1e-11 * sc)


def test_m0_r0_is_block_jacobi_schur_preconditioner():
    """m = 0, r = 0: S is replaced by C0 alone, so M is the block-triangular
    factorisation [[B, 0], [F, C0]] [[I, B^{-1}E], [0, I]] with the interface
    block solved block-diagonally (the plain block-diagonal Schur preconditioner)."""
    w, o, D, Es = _ops("lap", (12, 10), (3, 2), 1)
    o.set_lowrank(0, None, None)
    p, q = o.p, o.q
    Mfwd = np.block([[D["B"], np.zeros((p, q))], [D["F"], D["C0"]]]) @ \
        np.block([[np.eye(p), np.linalg.solve(D["B"], D["E"])], [np.zeros((q, p)), np.eye(q)]])
    _, _, perm = o.maps()
    b = np.random.default_rng(0).uniform(-1, 1, o.n)
    z = o.apply(b)
    zp = z[perm]
    np.testing.assert_allclose(Mfwd @ zp, b[perm], atol=1e-11)


def test_exact_full_rank_is_exact_inverse():
    """Exact local factors and r = q: S_app^{-1} = S^{-1} (Eq. 3.15 with
    V H V^T = E_rr), so M^{-1} = A^{-1} and FGMRES stops after one step."""
    w = C.lap2d_32_2x2_exact()
    o = O.from_workload(w)
    k, st = o.build_lowrank(w["m"], o.q, seed=0, full_rank=True)
    assert k == o.q
    b, xs = G.uniform_rhs(w["A"], 0)
    z = o.apply(b)
    np.testing.assert_allclose(z, xs, atol=1e-9)
    x, its, rel, st = o.fgmres(b)
    assert st == O.OK and its == 1 and rel <= 1e-8


def test_transpose_dot_product():
    w, o, D, Es = _ops("cd", (6, 6, 6), (3, 2, 1), 0)
    o.build_lowrank(3, 6, seed=2)
    rng = np.random.default_rng(5)
    for _ in range(3):
        u, v = rng.uniform(-1, 1, o.n), rng.uniform(-1, 1, o.n)
        a, b = o.apply(u) @ v, u @ o.apply_T(v)
        assert abs(a - b) <= 1e-13 * max(abs(a), 1.0) * 10


def test_prop3_and_spectral_similarity():
    """Proposition of Sec. 3.2.1 (Eq. 3.20-3.21): ||S^{-1} - S_app^{-1}|| / ||S^{-1}||
    <= ||X|| ||Z^{-1}|| (Frobenius), and Eq. 3.23: lambda(S_app^{-1} S) =
    1 - lambda(Z^{-1} X)."""
    w, o, D, Es = _ops("lap", (12, 10), (3, 2), 1)
    m, r = 3, 6
    o.build_lowrank(m, r, seed=0)
    V, H, Gm = o.lowrank()
    q = o.q
    S = D["C"] - D["F"] @ np.linalg.solve(D["B"], D["E"])
    Err = _columns(lambda v: o.Err(m, v), q)
    Pm = _columns(lambda v: o.series(m, v), q)
    Sapp = Pm @ (np.eye(q) + V @ Gm @ V.T)
    X = Err - V @ H @ V.T
    Z = np.eye(q) - V @ H @ V.T
    Si = np.linalg.inv(S)
    lhs = np.linalg.norm(Si - Sapp, "fro") / np.linalg.norm(Si, "fro")
    assert lhs <= np.linalg.norm(X, "fro") * np.linalg.norm(np.linalg.inv(Z), "fro")
    ev1 = np.sort_complex(np.linalg.eigvals(Sapp @ S))
    ev2 = np.sort_complex(1 - np.linalg.eigvals(np.linalg.solve(Z, X)))
    np.testing.assert_allclose(ev1, ev2, atol=1e-8)


def test_fgmres_unpreconditioned_distinct_eigenvalues():
    """GMRES on a diagonalizable matrix with k distinct eigenvalues terminates in
    at most k steps; a diagonal matrix with 3 values and a generic b takes
    exactly 3.  The oracle's A enters only through the CSR it is given."""
    n = 30
    d = np.array([1.0, 2.0, 5.0])[np.arange(n) % 3]
    A = G.CSR(n, np.arange(n + 1), np.arange(n), d)
    o = O.Oracle(A, dims=(n, 1, 1), splits=(1, 1, 1))
    b = np.random.default_rng(0).uniform(-1, 1, n)
    x, its, rel, st = o.fgmres(b, precond=False, rtol=1e-12)
    assert st == O.OK and its == 3
    np.testing.assert_allclose(x, b / d, atol=1e-12)


@pytest.mark.parametrize("transpose", [False, True])
def test_fgmres_solves_to_rtol(transpose):
    w = C.small_problem("cd", (8, 8, 8), (2, 2, 2), factor=0, m=3, rank=8, K=4)
    o = O.from_workload(w)
    o.build_lowrank(3, 8, seed=0)
    b, xs = G.uniform_rhs(w["A"], 0)
    D = G.dense_from_csr(w["A"])
    Ad = D.T if transpose else D
    x, its, rel, st = o.fgmres(b, rtol=1e-10, transpose=transpose)
    assert st == O.OK
    assert np.linalg.norm(b - Ad @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001
    xt = np.linalg.solve(Ad, b)
    # forward error bound: ||x - x*|| / ||x*|| <= cond(A) * relative residual
    assert np.linalg.norm(x - xt) <= 2 * np.linalg.cond(Ad) * 1e-10 * np.linalg.norm(xt)


def test_fgmres_restart_and_maxit():
    """Restarted GMRES converges for a positive definite matrix (Saad, Iterative
    Methods, Sec. 6.11.4); the iteration count runs across restarts and stops at
    maxit with a not-converged status."""
    n = 60
    d = 1.0 + np.arange(n, dtype=float)
    A = G.CSR(n, np.arange(n + 1), np.arange(n), d)
    o = O.Oracle(A, dims=(n, 1, 1), splits=(1, 1, 1))
    b = np.random.default_rng(0).uniform(-1, 1, n)
    x, its, rel, st = o.fgmres(b, precond=False, restart=5, maxit=12)
    assert st == O.ERR_NOT_CONVERGED and its == 12
    x, its2, rel2, st2 = o.fgmres(b, precond=False, restart=5, maxit=5000, rtol=1e-8)
    assert st2 == O.OK and rel2 <= 1e-8 and its2 > 5
    np.testing.assert_allclose(x, b / d, atol=1e-7)
    x, its3, rel3, st3 = o.fgmres(np.zeros(o.n))
    assert st3 == O.OK and its3 == 0 and not x.any()
