"""GPU checks of the two layouts of the triangular-sweep segments
(pslr_opts.merge_levels): one level of a factor per streamed segment, or
several consecutive levels per segment.  The layout changes only the copies
that feed the sweeps, never the arithmetic of a row, so a merged context must
reproduce a one-level context bit for bit: the apply of Algorithm 3 and its
transpose in both precisions, the E_rr(m) matvecs of the Arnoldi set-up (same
V, H and G), FGMRES, and the batched form.  Both stay within 1e-12 of the
oracle in FP64."""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12

CASES = [
    ("lap", (32, 32), (2, 2), 1),          # exact local LU with row pivots
    ("lap", (13, 11, 9), (3, 2, 2), 0),
    ("cd", (12, 10, 8), (3, 2, 2), 0),
    ("kappa", (10, 9, 11), (2, 3, 2), 0),
    ("lap", (13, 11, 9), (3, 2, 2), 2),    # ILUT(1e-2): general rows
    ("cd", (9, 9, 9), (1, 1, 1), 0),       # one subdomain, no interface
    ("lap", (7, 6, 5), (7, 6, 5), 0),      # one node per part, empty B
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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _pair(w):
    from paper_2002_00917_gb300 import pslr

    a = pslr.from_workload(w, merge_levels=1)
    b = pslr.from_workload(w, merge_levels=2)
    assert a.info["merged"] == [0, 0] and b.info["merged"] == [1, 1]
    return a, b


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_merged_layout_is_bit_exact(dev, case):
    kind, dims, splits, factor = case
    w = C.small_problem(kind, dims, splits, factor=factor, m=3, rank=6, K=3, drop_tol=1e-2)
    a, b = _pair(w)
    ra, _ = a.build_lowrank(3, 6)
    rb, _ = b.build_lowrank(3, 6)
    assert ra == rb
    for x, y in zip(a.get_lowrank(), b.get_lowrank()):
        assert np.array_equal(x, y)
    V, H, Gm = a.get_lowrank()
    orc = O.from_workload(w)
    orc.set_lowrank(3, V if ra else None, Gm if ra else None)
    rng = np.random.default_rng(21)
    for tr in (False, True):
        rhs = rng.uniform(-1, 1, w["A"].n)
        for dt in (torch.float64, torch.float32):
            bd = torch.tensor(rhs, device=dev, dtype=dt)
            za, zb = torch.full_like(bd, float("nan")), torch.full_like(bd, float("nan"))
            a.apply(bd, za, transpose=tr)
            b.apply(bd, zb, transpose=tr)
            a.sync()
            b.sync()
            assert torch.equal(za, zb), (tr, dt)
            if dt == torch.float64:
                ref = orc.apply_T(rhs) if tr else orc.apply(rhs)
                assert _rel(zb.cpu().numpy(), ref) <= TOL64, tr
    a.close()
    b.close()


def test_merged_layout_fgmres_is_bit_exact(dev):
    from paper_2002_00917_gb300 import pslr

    w = C.small_problem("lap", (24, 20, 16), (2, 2, 2), factor=0, m=3, rank=8, K=3)
    a, b = _pair(w)
    for c in (a, b):
        c.build_lowrank(3, 8)
    rhs = np.random.default_rng(5).uniform(-1, 1, w["A"].n)
    for prec in (pslr.PSLR_FP64, pslr.PSLR_FP32):
        out = []
        for c in (a, b):
            bd = torch.tensor(rhs, device=dev)
            x = torch.zeros_like(bd)
            its, rel, st = c.solve(bd, x, rtol=1e-8, restart=40, maxit=500, prec=prec)
            assert st == pslr.PSLR_OK
            out.append((its, rel, x.cpu().numpy()))
        assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
        assert np.array_equal(out[0][2], out[1][2])
    a.close()
    b.close()


def test_merged_systems_in_a_batch(dev):
    """The batched kernel sweeps a merged context's levels one barrier step
    each, as for a one-level context: the same result, bit for bit."""
    from paper_2002_00917_gb300 import pslr

    specs = [("lap", (20, 17), (3, 2), 3, 6), ("cd", (9, 8, 7), (2, 2, 2), 2, 5), ("lap", (12, 12), (2, 2), 0, 0)]
    plain, merged = [], []
    for kind, dims, splits, m, r in specs:
        w = C.small_problem(kind, dims, splits, m=m, rank=r, K=3)
        a, b = _pair(w)
        if r:
            orc = O.from_workload(w)
            orc.build_lowrank(m, r, seed=0)
            V, H, Gm = orc.lowrank()
            a.set_lowrank(m, V, Gm)
            b.set_lowrank(m, V, Gm)
        else:
            a.set_lowrank(m)
            b.set_lowrank(m)
        plain.append(a)
        merged.append(b)
    for nrhs in (1, 3):
        ba, bb = pslr.Batch(plain, nrhs), pslr.Batch(merged, nrhs)
        rhs = torch.tensor(np.random.default_rng(nrhs).uniform(-1, 1, ba.info["n_total"]), device=dev)
        for dt in (torch.float64, torch.float32):
            bd = rhs.to(dt)
            za, zb = torch.zeros_like(bd), torch.zeros_like(bd)
            ba.apply(bd, za)
            bb.apply(bd, zb)
            ba.sync()
            bb.sync()
            assert torch.equal(za, zb), (nrhs, dt)
        ba.close()
        bb.close()
    for c in plain + merged:
        c.close()


def test_full_size_merged_fp64_equals_one_level(dev):
    """128^3 convection-diffusion, 256 subdomains on two CTAs per SM: the
    automatic layout merges the FP64 sweeps; it must equal the one-level
    layout bit for bit in both directions and precisions (random low-rank
    term of rank 16, set on both)."""
    from paper_2002_00917_gb300 import pslr

    w = C.WORKLOADS["cd3d_128_8x8x4_ilu0"]()
    a = pslr.from_workload(w, merge_levels=1)
    b = pslr.from_workload(w)
    assert a.info["merged"] == [0, 0] and b.info["merged"] == [1, 0]
    assert b.info["ctas_per_sm"] == [2, 2]
    rng = np.random.default_rng(3)
    q = a.info["q"]
    V = np.linalg.qr(rng.standard_normal((q, 16)))[0]
    Gm = rng.uniform(-0.1, 0.1, (16, 16))
    for c in (a, b):
        c.set_lowrank(w["m"], V, Gm)
    rhs = rng.uniform(-1, 1, w["A"].n)
    for tr in (False, True):
        for dt in (torch.float64, torch.float32):
            bd = torch.tensor(rhs, device=dev, dtype=dt)
            za, zb = torch.zeros_like(bd), torch.zeros_like(bd)
            a.apply(bd, za, transpose=tr)
            b.apply(bd, zb, transpose=tr)
            a.sync()
            b.sync()
            assert torch.equal(za, zb), (tr, dt)
    a.close()
    b.close()
