"""GPU parity of the classical Neumann polynomial of Sec. 1 (pslr_set_neumann):
S^{-1} ~ omega [I + N + ... + N^m] D^{-1}, N = I - omega D^{-1} S, D = C0,
inside Algorithm 3's block elimination, against the oracle's restatement.

Bars as for the PSLR apply: FP64 within 1e-12 relative (2-norm and max-norm),
FP32 within 1e-5 (no low-rank term, so the FP32 form differs from the FP64
oracle only by its arithmetic), FGMRES iteration counts within +-1."""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5

CASES = [
    ("lap", (32, 32), (2, 2), 1),          # exact local LU with row pivots
    ("lap", (13, 11, 9), (3, 2, 2), 0),
    ("cd", (12, 10, 8), (3, 2, 2), 0),
    ("kappa", (10, 9, 11), (2, 3, 2), 0),
    ("lap", (13, 11, 9), (3, 2, 2), 2),    # ILUT(1e-2)
]
IDS = [f"{c[0]}{'x'.join(map(str, c[1]))}_f{c[3]}" for c in CASES]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build

    build.build()
    return torch.device("cuda:0")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


def _pair(case):
    from paper_2002_00917_gb300 import pslr

    kind, dims, splits, factor = case
    w = C.small_problem(kind, dims, splits, factor=factor, m=3, rank=0, K=3)
    return w, pslr.from_workload(w), O.from_workload(w)


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("m,omega", [(0, 0.7), (3, 0.6), (3, 1.4), (5, 0.9)])
def test_neumann_apply_matches_oracle(dev, case, m, omega):
    w, ctx, orc = _pair(case)
    ctx.set_neumann(m, omega)
    assert ctx.info["omega"] == omega and ctx.info["rank"] == 0 and ctx.info["m"] == m
    rng = np.random.default_rng(8)
    for tr in (False, True):
        b = rng.uniform(-1, 1, w["A"].n)
        zo = orc.neumann_apply(m, omega, b, transpose=tr)
        for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
            bd = torch.tensor(b, device=dev, dtype=dt)
            zd = torch.full_like(bd, float("nan"))
            ctx.apply(bd, zd, transpose=tr)
            ctx.sync()
            r2, rinf = _rel(zd.cpu().double().numpy(), zo)
            assert r2 <= tol and rinf <= tol, (tr, dt, r2, rinf)
    ctx.close()


@pytest.mark.parametrize("case", CASES[1:3], ids=IDS[1:3])
def test_omega_one_is_pslr_rank_zero_bit_for_bit(dev, case):
    """omega = 1 runs the PSLR code path unchanged: the result equals
    Algorithm 3 with no low-rank term exactly, in both precisions and both
    directions; and a new low-rank term returns the context to PSLR."""
    w, ctx, orc = _pair(case)
    rng = np.random.default_rng(1)
    for dt in (torch.float64, torch.float32):
        for tr in (False, True):
            bd = torch.tensor(rng.uniform(-1, 1, w["A"].n), device=dev, dtype=dt)
            za, zb = torch.zeros_like(bd), torch.zeros_like(bd)
            ctx.set_lowrank(3)
            ctx.apply(bd, za, transpose=tr)
            ctx.set_neumann(3, 1.0)
            ctx.apply(bd, zb, transpose=tr)
            ctx.sync()
            assert torch.equal(za, zb), (dt, tr)
    ctx.set_neumann(2, 0.5)
    k, _ = ctx.build_lowrank(3, 6)
    assert ctx.info["omega"] == 1.0
    V, H, Gm = ctx.get_lowrank()
    orc.set_lowrank(3, V, Gm)
    b = rng.uniform(-1, 1, w["A"].n)
    bd = torch.tensor(b, device=dev)
    zd = torch.zeros_like(bd)
    ctx.apply(bd, zd)
    ctx.sync()
    assert _rel(zd.cpu().numpy(), orc.apply(b))[0] <= TOL64
    ctx.close()


@pytest.mark.parametrize("omega", [0.8, 1.2])
def test_neumann_fgmres_iterations_match_oracle(dev, omega):
    """FGMRES preconditioned by the polynomial: iteration counts within one of
    the oracle's, and the true residual meets the tolerance."""
    from paper_2002_00917_gb300 import pslr

    w, ctx, orc = _pair(("lap", (24, 20, 16), (2, 2, 2), 0))
    m = 3
    ctx.set_neumann(m, omega)
    orc.set_neumann(m, omega)
    b, _ = G.uniform_rhs(w["A"], 0)
    _, its_o, rel_o, st_o = orc.fgmres(b, rtol=1e-8, restart=40, maxit=500)
    bd = torch.tensor(b, device=dev)
    x = torch.zeros_like(bd)
    its, rel, st = ctx.solve(bd, x, rtol=1e-8, restart=40, maxit=500)
    assert st_o == O.OK and st == pslr.PSLR_OK
    assert abs(its - its_o) <= 1, (its, its_o)
    r = b - G.csr_matvec(w["A"], x.cpu().numpy())
    assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(b)
    ctx.close()


def test_neumann_full_size_apply(dev):
    """The 64^3 workload's operators with the polynomial (m = 3, omega = 0.8),
    element by element against the oracle, both precisions."""
    from paper_2002_00917_gb300 import pslr

    w = C.lap3d_64_4x4x2_ilu0()
    ctx = pslr.from_workload(w)
    orc = O.from_workload(w)
    ctx.set_neumann(3, 0.8)
    b = np.random.default_rng(6).uniform(-1, 1, w["A"].n)
    zo = orc.neumann_apply(3, 0.8, b)
    for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        bd = torch.tensor(b, device=dev, dtype=dt)
        zd = torch.zeros_like(bd)
        ctx.apply(bd, zd)
        ctx.sync()
        r2, rinf = _rel(zd.cpu().double().numpy(), zo)
        assert r2 <= tol and rinf <= tol, (dt, r2, rinf)
    ctx.close()


def test_batch_rejects_a_neumann_context(dev):
    from paper_2002_00917_gb300 import pslr

    w, ctx, orc = _pair(CASES[1])
    ctx.set_neumann(2, 0.7)
    with pytest.raises(pslr.PslrError) as e:
        pslr.Batch([ctx], 1)
    assert e.value.status == pslr.PSLR_ERR_STATE
    ctx.close()


def test_bad_neumann_arguments(dev):
    from paper_2002_00917_gb300 import pslr

    w, ctx, orc = _pair(CASES[1])
    for m, omega in ((-1, 0.5), (2, 0.0), (2, -1.0), (2, float("inf")), (2, float("nan"))):
        with pytest.raises(pslr.PslrError) as e:
            ctx.set_neumann(m, omega)
        assert e.value.status == pslr.PSLR_ERR_ARG
    ctx.close()
