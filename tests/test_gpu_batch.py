"""GPU parity of the batched form: many uneven systems, several right-hand
sides each, in one launch per apply and one FGMRES per (system, rhs) pair.

The oracle has no batched form: a batch is a set of independent systems, so
the reference for problem (k, j) is the oracle's apply / FGMRES on system k
and right-hand side j.  Bars as for the single-system path: FP64 applies
within 1e-12, FP32 applies within 1e-5 (against the oracle on the same BF16
V), FGMRES iteration counts within +-1 of the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from pslr_inputs import configs as C
from pslr_inputs import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5

# (kind, dims, splits, m, r): uneven sizes, 2D and 3D, degenerate m = 0 / r = 0
SYSTEMS = [
    ("lap", (20, 17), (3, 2), 3, 6),
    ("lap", (33, 30), (4, 4), 2, 8),
    ("cd", (9, 8, 7), (2, 2, 2), 4, 5),
    ("lap", (12, 12), (2, 2), 0, 0),
    ("kappa", (8, 9, 7), (2, 2, 1), 1, 0),
    ("lap", (26, 19), (4, 3), 5, 12),
]
# degenerate systems: one subdomain (no interface, q = 0), one node per part (B empty, p = 0)
DEGENERATE = [
    ("cd", (9, 9, 9), (1, 1, 1), 3, 0),
    ("lap", (7, 6, 5), (7, 6, 5), 2, 3),
    ("lap", (15, 11), (3, 2), 1, 4),
]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build

    build.build()
    return torch.device("cuda:0")


def _bf16(x):
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb, np.abs(a - b).max() / np.abs(b).max()


def _system(spec, bf16_oracle=False):
    """A context and an oracle with the same low-rank term (the oracle's)."""
    from paper_2002_00917_gb300 import pslr

    kind, dims, splits, m, r = spec
    w = C.small_problem(kind, dims, splits, m=m, rank=r, K=3)
    ctx = pslr.from_workload(w)
    orc = O.from_workload(w)
    if r:
        orc.build_lowrank(m, r, seed=0)
        V, H, Gm = orc.lowrank()
        ctx.set_lowrank(m, V, Gm)
        if bf16_oracle:
            orc.set_lowrank(m, _bf16(V), Gm.astype(np.float32).astype(np.float64))
    else:
        ctx.set_lowrank(m)
        orc.set_lowrank(m, None, None)
    return w, ctx, orc


def _systems(specs, bf16_oracle=False):
    return [_system(s, bf16_oracle) for s in specs]


def _split(bt, v):
    """Batched vector -> list over systems of (n_k, nrhs) arrays."""
    out = []
    for p, o in zip(bt.systems, bt.offsets()):
        out.append(v[o:o + p.n * bt.nrhs].reshape(bt.nrhs, p.n).T)
    return out


@pytest.mark.parametrize("nrhs", [1, 3, 4])
def test_batch_apply_fp64_matches_oracle(dev, nrhs):
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS)
    bt = pslr.Batch([c for _, c, _ in sy], nrhs)
    N = bt.info["n_total"]
    assert N == sum(w["A"].n for w, _, _ in sy) * nrhs
    b = np.random.default_rng(11).uniform(-1, 1, N)
    bd = torch.tensor(b, device=dev)
    zd = torch.full_like(bd, np.nan)
    bt.apply(bd, zd)
    bt.sync()
    z = zd.cpu().numpy()
    for (w, ctx, orc), bk, zk in zip(sy, _split(bt, b), _split(bt, z)):
        for j in range(nrhs):
            r2, rinf = _rel(zk[:, j], orc.apply(np.ascontiguousarray(bk[:, j])))
            assert r2 <= TOL64 and rinf <= TOL64, (w["A"].n, j, r2, rinf)


@pytest.mark.parametrize("group", [0, 1, 2, 3, 8])
def test_batch_apply_equals_single_system_apply(dev, group):
    """The batched launch and the per-system launches run the same arithmetic
    per row, whatever number of subdomains a CTA sweeps in lockstep (merged
    levels); only the order of the low-rank partial sums could differ."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS)
    bt = pslr.Batch([c for _, c, _ in sy], 2, group=group)
    if group:
        assert max(bt.info["group"]) <= group
    b = torch.tensor(np.random.default_rng(12).uniform(-1, 1, bt.info["n_total"]), device=dev)
    z = torch.zeros_like(b)
    bt.apply(b, z)
    bt.sync()
    for (w, ctx, _), o in zip(sy, bt.offsets()):
        n = w["A"].n
        bk = b[o:o + 2 * n].reshape(2, n).T  # column-major (n, 2) view
        zk = torch.zeros_like(bk)
        ctx.apply(bk, zk)
        ctx.sync()
        r2, rinf = _rel(z[o:o + 2 * n].reshape(2, n).T.cpu().numpy(), zk.cpu().numpy())
        assert r2 <= 1e-14 and rinf <= 1e-14, (n, r2, rinf)


def test_batch_apply_fp32_matches_oracle(dev):
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS, bf16_oracle=True)
    bt = pslr.Batch([c for _, c, _ in sy], 4)
    b = np.random.default_rng(13).uniform(-1, 1, bt.info["n_total"]).astype(np.float32)
    bd = torch.tensor(b, device=dev)
    zd = torch.zeros_like(bd)
    bt.apply(bd, zd)
    bt.sync()
    z = zd.cpu().double().numpy()
    for (w, ctx, orc), bk, zk in zip(sy, _split(bt, b.astype(np.float64)), _split(bt, z)):
        for j in range(4):
            r2, rinf = _rel(zk[:, j], orc.apply(np.ascontiguousarray(bk[:, j])))
            assert r2 <= TOL32 and rinf <= TOL32, (w["A"].n, j, r2, rinf)


@pytest.mark.parametrize("group", [1, 0])
def test_batch_more_items_than_ctas(dev, group):
    """40 systems of 16 subdomains: several groups per CTA in every phase, with
    m and r varying across systems."""
    from paper_2002_00917_gb300 import pslr

    specs = [("lap", (16 + (k % 7), 16 + (k % 5)), (4, 4), k % 4, (0, 4, 8)[k % 3]) for k in range(40)]
    sy = _systems(specs)
    bt = pslr.Batch([c for _, c, _ in sy], 2, group=group)
    assert bt.info["items"] == 640
    if group == 1:
        assert bt.info["groups"] == [640, 640] and bt.info["grid"] < 640
    b = np.random.default_rng(14).uniform(-1, 1, bt.info["n_total"])
    bd = torch.tensor(b, device=dev)
    zd = torch.zeros_like(bd)
    bt.apply(bd, zd)
    bt.sync()
    for (w, ctx, orc), bk, zk in zip(sy, _split(bt, b), _split(bt, zd.cpu().numpy())):
        for j in range(2):
            r2, rinf = _rel(zk[:, j], orc.apply(np.ascontiguousarray(bk[:, j])))
            assert r2 <= TOL64 and rinf <= TOL64


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_batch_solve(dev, prec):
    """Every (system, rhs) problem converges to 1e-8 in its true residual; in
    FP64 its iteration count is within +-1 of the oracle's FGMRES."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS)
    nrhs = 3
    bt = pslr.Batch([c for _, c, _ in sy], nrhs)
    rng = np.random.default_rng(15)
    bs = []
    for w, _, _ in sy:
        cols = [G.csr_matvec(w["A"], rng.uniform(-1, 1, w["A"].n)) for _ in range(nrhs)]
        bs.append(np.concatenate(cols))
    b = np.concatenate(bs)
    bd = torch.tensor(b, device=dev)
    x = torch.zeros_like(bd)
    # a first solve with other limits: the cycle graph it captures serves the next one
    its1, _, st1 = bt.solve(bd, x, rtol=1e-3, restart=20, maxit=1, prec=prec)
    assert st1 in (pslr.PSLR_OK, pslr.PSLR_ERR_NOT_CONVERGED) and np.all(its1 == 1)
    its, rel, st = bt.solve(bd, x, rtol=1e-8, restart=20, maxit=400, prec=prec)
    assert st == pslr.PSLR_OK, (its, rel)
    assert bt.info["graph"] == 1
    xs = _split(bt, x.cpu().numpy())
    for k, ((w, ctx, orc), bk) in enumerate(zip(sy, _split(bt, b))):
        A = G.dense_from_csr(w["A"])
        for j in range(nrhs):
            p = k * nrhs + j
            assert rel[p] <= 1e-8
            assert np.linalg.norm(bk[:, j] - A @ xs[k][:, j]) <= 1.0001e-8 * np.linalg.norm(bk[:, j])
            if prec == 0:
                _, its_o, _, st_o = orc.fgmres(np.ascontiguousarray(bk[:, j]), rtol=1e-8, restart=20, maxit=400)
                assert st_o == 0 and abs(int(its[p]) - its_o) <= 1, (k, j, its[p], its_o)



@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_batch_solve_finishes_stragglers_per_system(dev, prec):
    """Once at most 16 of more than 16 problems still run at a cycle end, they
    are finished on their own systems (pslr_solve on the current residual,
    systems in parallel threads).  Six test systems with three rhs each (18
    problems) at restart 20; the oracle's counts say whether that happens
    (the oracle needs 35-90 iterations on these systems); the batch must then
    report the hand-offs, meet the tolerance in every true residual and, in
    FP64, keep every iteration count within +-1 of the oracle's."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS)
    nrhs = 3
    bt = pslr.Batch([c for _, c, _ in sy], nrhs)
    rng = np.random.default_rng(25)
    bs = [[G.csr_matvec(w["A"], rng.uniform(-1, 1, w["A"].n)) for _ in range(nrhs)] for w, _, _ in sy]
    b = np.concatenate([np.concatenate(c) for c in bs])
    bd = torch.tensor(b, device=dev)
    x = torch.zeros_like(bd)
    restart = 20
    its, rel, st = bt.solve(bd, x, rtol=1e-8, restart=restart, maxit=2000, prec=prec)
    assert st == pslr.PSLR_OK, (its, rel)
    its_o = [orc.fgmres(bj, rtol=1e-8, restart=restart, maxit=2000)[1] for (w, c, orc), bk in zip(sy, bs) for bj in bk]
    # cycle ends at multiples of the restart: a hand-off happens at the first
    # one where 1..16 problems still need more iterations
    ends = range(restart, max(its_o) + restart, restart)
    expect = any(0 < sum(i > e for i in its_o) <= 16 for e in ends)
    if prec == 0:
        assert all(abs(int(a) - o) <= 1 for a, o in zip(its, its_o)), (its, its_o)
    if expect:
        assert bt.info["handoff"] >= 1
    xs = _split(bt, x.cpu().numpy())
    for k, ((w, _, _), bk) in enumerate(zip(sy, bs)):
        for j in range(nrhs):
            assert rel[k * nrhs + j] <= 1e-8
            r = bk[j] - G.csr_matvec(w["A"], xs[k][:, j])
            assert np.linalg.norm(r) <= 1.0001e-8 * np.linalg.norm(bk[j]), (k, j)



def test_batch_solve_handoff_reaches_maxit(dev):
    """Problems finished on their own systems keep the batch's iteration
    limit: with maxit 60 (restart 20) the six problems still running after
    two cycles are handed off with 20 iterations left; they stop at exactly
    60, the call reports PSLR_ERR_NOT_CONVERGED, and every returned relative
    residual is the true one of the returned x."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS)
    nrhs = 3
    bt = pslr.Batch([c for _, c, _ in sy], nrhs)
    rng = np.random.default_rng(26)
    bs = [[G.csr_matvec(w["A"], rng.uniform(-1, 1, w["A"].n)) for _ in range(nrhs)] for w, _, _ in sy]
    bd = torch.tensor(np.concatenate([np.concatenate(c) for c in bs]), device=dev)
    x = torch.zeros_like(bd)
    its, rel, st = bt.solve(bd, x, rtol=1e-8, restart=20, maxit=60, check=False)
    assert st == pslr.PSLR_ERR_NOT_CONVERGED
    assert np.all(its <= 60)
    stopped = its == 60
    assert stopped.any() and np.all(rel[stopped] > 1e-8)
    assert bt.info["handoff"] >= 1
    xs = _split(bt, x.cpu().numpy())
    for k, ((w, _, _), bk) in enumerate(zip(sy, bs)):
        for j in range(nrhs):
            r = np.linalg.norm(bk[j] - G.csr_matvec(w["A"], xs[k][:, j])) / np.linalg.norm(bk[j])
            assert abs(r - rel[k * nrhs + j]) <= 1e-6 * max(r, 1e-12) + 1e-14, (k, j, r, rel[k * nrhs + j])


def test_batch_apply_ilut_systems(dev):
    """Systems factored by ILUT(1e-2) (wider rows, fill) in a batch with an
    ILU(0) one: every (system, rhs) equals its oracle apply (FP64, 1e-12)."""
    from paper_2002_00917_gb300 import pslr

    specs = [("lap", (20, 17), (3, 2), 3, 6, 2), ("cd", (9, 8, 7), (2, 2, 2), 2, 5, 2),
             ("lap", (26, 19), (4, 3), 2, 8, 0)]
    sy = []
    for kind, dims, splits, m, r, factor in specs:
        w = C.small_problem(kind, dims, splits, factor=factor, m=m, rank=r, K=3)
        ctx = pslr.from_workload(w)
        orc = O.from_workload(w)
        orc.build_lowrank(m, r, seed=0)
        V, H, Gm = orc.lowrank()
        ctx.set_lowrank(m, V, Gm)
        sy.append((w, ctx, orc))
    nrhs = 2
    bt = pslr.Batch([c for _, c, _ in sy], nrhs)
    b = np.random.default_rng(31).uniform(-1, 1, bt.info["n_total"])
    bd = torch.tensor(b, device=dev)
    zd = torch.full_like(bd, np.nan)
    bt.apply(bd, zd)
    bt.sync()
    zs, bs = _split(bt, zd.cpu().numpy()), _split(bt, b)
    for (w, _, orc), zk, bk in zip(sy, zs, bs):
        for j in range(nrhs):
            ref = orc.apply(np.ascontiguousarray(bk[:, j]))
            assert np.linalg.norm(zk[:, j] - ref) <= 1e-12 * np.linalg.norm(ref), w["name"]


def test_batch_solve_maxit_and_zero_rhs(dev):
    """A zero right-hand side is solved by x = 0 in 0 iterations; the others
    stop at maxit and the call reports PSLR_ERR_NOT_CONVERGED."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS[:3])
    bt = pslr.Batch([c for _, c, _ in sy], 2)
    b = np.random.default_rng(16).uniform(-1, 1, bt.info["n_total"])
    o = bt.offsets()
    n1 = sy[1][0]["A"].n
    b[o[1]:o[1] + n1] = 0.0  # system 1, rhs 0
    bd = torch.tensor(b, device=dev)
    x = torch.zeros_like(bd)
    its, rel, st = bt.solve(bd, x, rtol=1e-14, restart=2, maxit=3)
    assert st == pslr.PSLR_ERR_NOT_CONVERGED
    assert its[2] == 0 and rel[2] == 0.0
    assert np.all(x[o[1]:o[1] + n1].cpu().numpy() == 0.0)
    assert all(its[p] == 3 for p in range(6) if p != 2)


def test_batch_rejects_stale_lowrank_and_bad_arguments(dev):
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS[:2])
    bt = pslr.Batch([c for _, c, _ in sy], 1)
    b = torch.zeros(bt.info["n_total"], device=dev, dtype=torch.float64)
    z = torch.zeros_like(b)
    sy[0][1].set_lowrank(1)  # replaces system 0's low-rank term
    with pytest.raises(pslr.PslrError) as e:
        bt.apply(b, z)
    assert e.value.status == pslr.PSLR_ERR_STATE
    with pytest.raises(pslr.PslrError) as e:
        pslr.Batch([c for _, c, _ in sy], 5)
    assert e.value.status == pslr.PSLR_ERR_ARG
    w = C.small_problem("lap", (10, 10), (2, 2), factor=1, K=3)
    exact = pslr.from_workload(w)
    exact.set_lowrank(1)
    with pytest.raises(pslr.PslrError) as e:
        pslr.Batch([exact], 1)
    assert e.value.status == pslr.PSLR_ERR_ARG


def test_batch_timeout_path_reports_and_recovers(dev):
    """A grid-barrier wait with limit 0 gives up at once; the batch reports
    PSLR_ERR_TIMEOUT and the next apply is correct.  No GPU fault is involved."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS[:3])
    bt = pslr.Batch([c for _, c, _ in sy], 2)
    b = np.random.default_rng(17).uniform(-1, 1, bt.info["n_total"])
    bd = torch.tensor(b, device=dev)
    zd = torch.zeros_like(bd)
    old = bt.set_wait_limit(0)
    bt.apply(bd, zd)
    assert bt.sync(check=False) == pslr.PSLR_ERR_TIMEOUT
    bt.set_wait_limit(old)
    bt.apply(bd, zd)
    bt.sync()
    for (w, ctx, orc), bk, zk in zip(sy, _split(bt, b), _split(bt, zd.cpu().numpy())):
        r2, _ = _rel(zk[:, 1], orc.apply(np.ascontiguousarray(bk[:, 1])))
        assert r2 <= TOL64


@pytest.mark.parametrize("group", [0, 1, 3])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_batch_degenerate_systems(dev, group, nrhs):
    """Systems without an interface or without interiors, mixed with a regular
    one, in every grouping: the batched apply still equals the oracle."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(DEGENERATE)
    bt = pslr.Batch([c for _, c, _ in sy], nrhs, group=group)
    b = np.random.default_rng(18).uniform(-1, 1, bt.info["n_total"])
    bd = torch.tensor(b, device=dev)
    zd = torch.full_like(bd, np.nan)
    bt.apply(bd, zd)
    bt.sync()
    for (w, ctx, orc), bk, zk in zip(sy, _split(bt, b), _split(bt, zd.cpu().numpy())):
        for j in range(nrhs):
            r2, rinf = _rel(zk[:, j], orc.apply(np.ascontiguousarray(bk[:, j])))
            assert r2 <= TOL64 and rinf <= TOL64, (w["A"].n, j, r2, rinf)


def test_autotune_group_picks_a_candidate_and_stays_exact(dev):
    """The group-size autotuner times each candidate and returns the fastest;
    the batch built with its choice still matches the oracle."""
    from paper_2002_00917_gb300 import autotune, pslr

    sy = _systems(SYSTEMS)
    ctxs = [c for _, c, _ in sy]
    best, table = autotune.tune_group(ctxs, 2, prec=pslr.PSLR_FP64, candidates=(1, 2, 0), steps=3, warmup=1)
    assert best in (1, 2, 0) and set(table) == {1, 2, 0}
    assert all(ms > 0 for _, ms in table.values())
    bt = pslr.Batch(ctxs, 2, group=best)
    b = np.random.default_rng(19).uniform(-1, 1, bt.info["n_total"])
    bd = torch.tensor(b, device=dev)
    zd = torch.zeros_like(bd)
    bt.apply(bd, zd)
    bt.sync()
    for (w, ctx, orc), bk, zk in zip(sy, _split(bt, b), _split(bt, zd.cpu().numpy())):
        for j in range(2):
            r2, rinf = _rel(zk[:, j], orc.apply(np.ascontiguousarray(bk[:, j])))
            assert r2 <= TOL64 and rinf <= TOL64


def test_launch_options_change_speed_not_results(dev):
    """pslr_batch_create_opts: the FP64 (row, rhs) mapping and a cap on the
    ring depth leave every applied value unchanged, bit for bit, in both
    precisions; per-precision group requests are honoured (reduced to fit)."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS)
    ctxs = [c for _, c, _ in sy]
    ref = pslr.Batch(ctxs, 3, group=(2, 4))
    assert ref.info["group"][0] <= 2 and ref.info["group"][1] <= 4 and ref.info["pair_rhs"] == 1
    b = torch.tensor(np.random.default_rng(23).uniform(-1, 1, ref.info["n_total"]), device=dev)
    outs = {}
    for key, kw in (("ref", None), ("rows", dict(pair_rhs=0)), ("ring3", dict(ring_max=(3, 3))),
                    ("both", dict(pair_rhs=0, ring_max=(2, 2)))):
        bt = ref if kw is None else pslr.Batch(ctxs, 3, group=(2, 4), **kw)
        if kw and "ring_max" in kw:
            assert bt.info["ring"][0] <= kw["ring_max"][0] and bt.info["ring"][1] <= kw["ring_max"][1]
        if kw and "pair_rhs" in kw:
            assert bt.info["pair_rhs"] == kw["pair_rhs"]
        res = []
        for dt in (torch.float64, torch.float32):
            bb = b.to(dt)
            z = torch.full_like(bb, float("nan"))
            bt.apply(bb, z)
            bt.sync()
            res.append(z)
        outs[key] = res
        if bt is not ref:
            bt.close()
    for key in ("rows", "ring3", "both"):
        for a, c in zip(outs["ref"], outs[key]):
            assert torch.equal(a, c), key
    ref.close()


def test_krylov_chunk_option_and_bad_options(dev):
    """A shorter Krylov chunk changes only the order of the per-problem
    partial sums: the batched FGMRES still reaches 1e-8 on every problem in
    about the same iterations.  Out-of-range options are rejected."""
    from paper_2002_00917_gb300 import pslr

    sy = _systems(SYSTEMS[:3])
    ctxs = [c for _, c, _ in sy]
    its = []
    for ch in (0, 256):
        bt = pslr.Batch(ctxs, 2, krylov_chunk=ch)
        assert bt.info["krylov_chunk"] == (ch or 1024)
        b = torch.tensor(np.random.default_rng(29).uniform(-1, 1, bt.info["n_total"]), device=dev)
        x = torch.zeros_like(b)
        it, rel, st = bt.solve(b, x, rtol=1e-8, restart=40, maxit=800)
        assert st == pslr.PSLR_OK and (rel <= 1e-8).all()
        its.append(it)
        bt.close()
    assert np.abs(its[0].astype(int) - its[1].astype(int)).max() <= 2, (its[0], its[1])
    for kw in (dict(ring_max=(1, 0)), dict(ring_max=(0, -1)), dict(krylov_chunk=32), dict(pair_rhs=2),
               dict(group=(9, 0)), dict(group=(0, -1))):
        with pytest.raises(pslr.PslrError) as e:
            pslr.Batch(ctxs, 2, **kw)
        assert e.value.status == pslr.PSLR_ERR_ARG, kw


def test_tune_batch_searches_every_knob(dev):
    """The autotuner times every apply candidate per precision and every
    Krylov chunk length, and returns options of the candidates it timed; a
    batch built with them matches the oracle."""
    from paper_2002_00917_gb300 import autotune, pslr

    sy = _systems(SYSTEMS)
    ctxs = [c for _, c, _ in sy]
    best, table = autotune.tune_batch(ctxs, 2, groups=((0, 2), (0, 4)), rings=(0, 3), pairs=(1, 0),
                                      chunks=(512, 1024), restart=20, maxit=200, steps=2, warmup=1)
    applies64 = [r for r in table if r["what"] == "apply_fp64"]
    applies32 = [r for r in table if r["what"] == "apply_fp32"]
    cycles = [r for r in table if r["what"].startswith("fgmres")]
    assert len(applies64) == 2 * 2 * 2 and len(applies32) == 2 * 2 and len(cycles) == 2
    assert all(r["ms"] > 0 for r in table)
    assert best["group"][0] in (0, 2) and best["group"][1] in (0, 4) and best["pair_rhs"] in (0, 1)
    assert best["krylov_chunk"] in (512, 1024) and all(v in (0, 3) for v in best["ring_max"])
    bt = pslr.Batch(ctxs, 2, **best)
    b = np.random.default_rng(31).uniform(-1, 1, bt.info["n_total"])
    bd = torch.tensor(b, device=dev)
    zd = torch.zeros_like(bd)
    bt.apply(bd, zd)
    bt.sync()
    for (w, ctx, orc), bk, zk in zip(sy, _split(bt, b), _split(bt, zd.cpu().numpy())):
        for j in range(2):
            r2, rinf = _rel(zk[:, j], orc.apply(np.ascontiguousarray(bk[:, j])))
            assert r2 <= TOL64 and rinf <= TOL64
    bt.close()
