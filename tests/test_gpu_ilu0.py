"""Device ILU(0) (Algorithm 1, steps 3-4 with ILU(0) local factors; Saad,
Iterative Methods, Sec. 10.3.2): pslr_ilu0_device against the oracle's
factors and against the defining property of ILU(0), and set-ups that factor
on the GPU (pslr_opts.device_factor) against the oracle's apply.

Bars: factor values within 1e-12 relative (2-norm and max-norm) of the
oracle's (the device fuses a_ij - l_ik u_kj into one rounding, so the two
differ by rounding only); (L U)_ij = a_ij on the pattern within 1e-12; FP64
applies within 1e-12 as in the other parity tests.
"""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def pslr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build, pslr

    build.build()
    return pslr


def _rel(a, b):
    if b.size == 0:
        return 0.0, 0.0
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


def _factor(pslr, bptr, rp, ci, v):
    val = torch.tensor(np.asarray(v, np.float64), device="cuda")
    pslr.ilu0_device(bptr, rp, ci, val)
    return val.cpu().numpy()


CASES = [
    ("lap", (32, 32), (2, 2)),
    ("lap", (13, 11, 9), (3, 2, 2)),
    ("cd", (12, 10, 8), (3, 2, 2)),
    ("kappa", (10, 9, 11), (2, 3, 2)),
    ("lap", (24, 20, 16), (2, 2, 2)),
    ("cd", (9, 9, 9), (1, 1, 1)),      # one subdomain: C0 empty
    ("lap", (7, 6, 5), (7, 6, 5)),     # every node its own part: B empty
]


@pytest.mark.parametrize("kind,dims,splits", CASES, ids=[f"{c[0]}{'x'.join(map(str, c[1]))}" for c in CASES])
def test_device_factor_equals_oracle_factor(pslr, kind, dims, splits):
    """B = blockdiag(B_i) and C0 = blockdiag(C_i) of the oracle's set-up,
    factored on the device block by block, against the oracle's ILU(0)."""
    o = O.from_workload(C.small_problem(kind, dims, splits, K=3))
    io, go = o.offsets()
    for blk, fac, bptr in (("B", "LU_B", io), ("C0", "LU_C0", go)):
        rp, ci, v, _ = o.block(blk)
        frp, fci, fv, _ = o.block(fac)
        np.testing.assert_array_equal(rp, frp)
        np.testing.assert_array_equal(ci, fci)
        got = _factor(pslr, bptr, rp, ci, v)
        r2, rinf = _rel(got, fv)
        assert r2 <= TOL and rinf <= TOL, (blk, r2, rinf)


def _random_blocks(sizes, seed):
    """A block-diagonal matrix with random nonsymmetric patterns (about 2-8
    entries per row, the diagonal always stored and made dominant, so ILU(0)
    exists), as host CSR."""
    rng = np.random.default_rng(seed)
    rp, ci, v, bptr = [0], [], [], [0]
    for nbk in sizes:
        r0 = bptr[-1]
        for i in range(nbk):
            k = int(rng.integers(1, 8))
            cols = set(rng.integers(0, nbk, k).tolist()) | {i}
            # also a near neighbour below the diagonal, so levels chain
            if i > 0 and rng.random() < 0.7:
                cols.add(i - 1)
            cols = sorted(cols)
            vals = rng.uniform(-1, 1, len(cols))
            vals[cols.index(i)] = len(cols) + 1.0 + rng.random()
            ci.extend(r0 + c for c in cols)
            v.extend(vals.tolist())
            rp.append(len(ci))
        bptr.append(r0 + nbk)
    return np.array(bptr), np.array(rp), np.array(ci), np.array(v)


@pytest.mark.parametrize("sizes", [[1], [5, 300, 1, 77], [1000], [40] * 200])
def test_ilu0_property_on_random_blocks(pslr, sizes):
    """ILU(0) is defined by (L U)_ij = a_ij for every (i, j) in the pattern of
    A, with L unit lower and U upper on that pattern (Saad, Sec. 10.3.2):
    checked densely per block, independently of the oracle.  Levels with more
    rows than a CTA has threads, and many blocks, are covered."""
    bptr, rp, ci, v = _random_blocks(sizes, seed=len(sizes))
    f = _factor(pslr, bptr, rp, ci, v)
    for b in range(len(sizes)):
        r0, r1 = bptr[b], bptr[b + 1]
        nbk = r1 - r0
        A = np.zeros((nbk, nbk))
        F = np.zeros((nbk, nbk))
        for i in range(r0, r1):
            for k in range(rp[i], rp[i + 1]):
                A[i - r0, ci[k] - r0] = v[k]
                F[i - r0, ci[k] - r0] = f[k]
        L = np.tril(F, -1) + np.eye(nbk)
        U = np.triu(F)
        pat = A != 0
        LU = L @ U
        err = np.abs(LU[pat] - A[pat]).max() / np.abs(A).max()
        assert err <= TOL, (b, err)


def test_ilu0_device_zero_pivot(pslr):
    """[[1, 1], [1, 1]]: u_11 = 1 - 1 * 1 = 0, reported as a zero pivot; a
    set-up whose local ILU(0) meets a zero pivot fails the same way."""
    with pytest.raises(pslr.PslrError) as e:
        _factor(pslr, [0, 2], [0, 2, 4], [0, 1, 0, 1], [1.0, 1.0, 1.0, 1.0])
    assert e.value.status == pslr.PSLR_ERR_ZERO_PIVOT
    A = G.shifted_laplacian((6, 5), 0.1)
    zp = G.CSR(A.n, A.rowptr, A.col, A.val.copy())
    zp.val[zp.rowptr[0]] = 0.0  # the diagonal of row 0
    with pytest.raises(pslr.PslrError) as e:
        pslr.Pslr(zp, dims=(6, 5, 1), splits=(2, 1, 1), device_factor=True)
    assert e.value.status == pslr.PSLR_ERR_ZERO_PIVOT


APPLY_CASES = [
    ("lap", (13, 11, 9), (3, 2, 2), 3, 6),
    ("cd", (12, 10, 8), (3, 2, 2), 2, 5),
    ("kappa", (10, 9, 11), (2, 3, 2), 4, 7),
    ("lap", (24, 20, 16), (2, 2, 2), 5, 16),
]


@pytest.mark.parametrize("kind,dims,splits,m,r", APPLY_CASES, ids=[f"{c[0]}{'x'.join(map(str, c[1]))}" for c in APPLY_CASES])
def test_setup_with_device_factor_apply_parity(pslr, kind, dims, splits, m, r):
    """A context whose local factors came from the device: forward and
    transposed FP64 applies against the oracle at 1e-12, and against the
    context that factored on the host."""
    w = C.small_problem(kind, dims, splits, m=m, rank=r, K=3)
    ctx = pslr.from_workload(w, device_factor=True)
    host = pslr.from_workload(w)
    orc = O.from_workload(w)
    assert ctx.info["device_factor"] == 1 and ctx.info["factor_ms"] > 0
    assert host.info["device_factor"] == 0
    assert ctx.info["nnz_ilu"] == host.info["nnz_ilu"]
    orc.build_lowrank(m, r, seed=0)
    V, H, Gm = orc.lowrank()
    ctx.set_lowrank(m, V, Gm)
    host.set_lowrank(m, V, Gm)
    b = np.random.default_rng(5).uniform(-1, 1, w["A"].n)
    bd = torch.tensor(b, device="cuda")
    for transpose in (False, True):
        z, zh = torch.zeros_like(bd), torch.zeros_like(bd)
        ctx.apply(bd, z, transpose=transpose)
        host.apply(bd, zh, transpose=transpose)
        ctx.sync()
        host.sync()
        zo = orc.apply_T(b) if transpose else orc.apply(b)
        for got in (z, zh):
            r2, rinf = _rel(got.cpu().numpy(), zo)
            assert r2 <= TOL and rinf <= TOL, (transpose, r2, rinf)
    ctx.close()
    host.close()


@pytest.mark.parametrize("name", ["lap3d_64_4x4x2_ilu0", "cd3d_128_8x8x4_ilu0"])
def test_device_factor_full_size(pslr, name):
    """At the bench's sizes: the device-factored context's FP64 apply equals
    the host-factored one's within 1e-12 (same factors up to rounding)."""
    w = C.WORKLOADS[name]()
    ctx = pslr.from_workload(w, device_factor=True)
    host = pslr.from_workload(w)
    assert ctx.info["device_factor"] == 1 and ctx.info["factor_ms"] > 0
    rng = np.random.default_rng(0)
    q, r = ctx.info["q"], w["rank"]
    V = np.linalg.qr(rng.standard_normal((q, r)))[0]
    Gm = rng.uniform(-0.01, 0.01, (r, r))
    ctx.set_lowrank(w["m"], V, Gm)
    host.set_lowrank(w["m"], V, Gm)
    bd = torch.tensor(rng.uniform(-1, 1, w["A"].n), device="cuda")
    z, zh = torch.zeros_like(bd), torch.zeros_like(bd)
    ctx.apply(bd, z)
    host.apply(bd, zh)
    ctx.sync()
    host.sync()
    r2, rinf = _rel(z.cpu().numpy(), zh.cpu().numpy())
    assert r2 <= TOL and rinf <= TOL, (r2, rinf)
    ctx.close()
    host.close()
