"""pslr_apply_noalloc: the apply for callers that cannot allocate device memory
when they apply the preconditioner (their device memory belongs to a pool
allocator of their own and cudaMalloc/cudaFree are off limits).  It runs the
same apply kernel with the same arguments on a scratch array that lives
inside the library instead of on buffers the context allocated, so its
result must equal pslr_apply's bit for bit.  This file is collected last on
purpose: a run that stops at its first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

from pslr_inputs import configs as Cf
from pslr_inputs import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build

    build.build()
    return torch.device("cuda:0")


def _workload():
    return Cf.small_problem("cd", (12, 10, 8), (3, 2, 2), factor=0, m=3, rank=6, K=3)


def _noalloc(lib, ctx, b, z, prec, transpose):
    from paper_2002_00917_gb300 import pslr

    return lib.pslr_apply_noalloc(ctx.h, C.c_void_p(b.data_ptr()), C.c_void_p(z.data_ptr()), prec,
                                  transpose, pslr._stream(None))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_apply_noalloc_equals_apply_twice(dev, prec):
    """Two calls in a row per direction (the shared array keeps the previous
    call's contents): each equals pslr_apply on the same input exactly."""
    from paper_2002_00917_gb300 import pslr

    w = _workload()
    ctx = pslr.from_workload(w)
    ctx.build_lowrank(w["m"], w["rank"])
    lib = pslr.load()
    dt = torch.float64 if prec == 0 else torch.float32
    rng = np.random.default_rng(11)
    for transpose in (0, 1):
        for call in range(2):
            b = torch.tensor(rng.uniform(-1, 1, w["A"].n), device=dev, dtype=dt)
            z_ref = torch.zeros_like(b)
            z_na = torch.full_like(b, float("nan"))
            ctx.apply(b, z_ref, transpose=bool(transpose))
            st = _noalloc(lib, ctx, b, z_na, prec, transpose)
            assert st == pslr.PSLR_OK, lib.pslr_last_error(ctx.h).decode()
            ctx.sync()
            assert np.array_equal(z_na.cpu().numpy(), z_ref.cpu().numpy()), (transpose, call)
    ctx.close()


def test_apply_noalloc_matches_oracle(dev):
    """The FP64 result against the FP64 oracle (Algorithm 3) on the same
    low-rank term, within the 1e-12 relative bar of the FP64 apply."""
    import oracle as O
    from paper_2002_00917_gb300 import pslr

    w = _workload()
    ctx = pslr.from_workload(w)
    ctx.build_lowrank(w["m"], w["rank"])
    V, H, Gm = ctx.get_lowrank()
    orc = O.from_workload(w)
    orc.set_lowrank(w["m"], V, Gm)
    lib = pslr.load()
    b = np.random.default_rng(5).uniform(-1, 1, w["A"].n)
    bd = torch.tensor(b, device=dev)
    for call in range(2):
        zd = torch.full_like(bd, float("nan"))
        assert _noalloc(lib, ctx, bd, zd, 0, 0) == pslr.PSLR_OK
        ctx.sync()
        zo = orc.apply(b)
        rel = np.linalg.norm(zd.cpu().numpy() - zo) / np.linalg.norm(zo)
        assert rel <= 1e-12, (call, rel)
    ctx.close()


def test_apply_noalloc_timeout_is_reported_and_recovers(dev):
    """A grid-barrier wait whose limit is 0 gives up at once: the error
    latches in the context's own error word, pslr_sync reports
    PSLR_ERR_TIMEOUT, and once the limit is back the next call is exact
    again.  No GPU fault is involved."""
    from paper_2002_00917_gb300 import pslr

    w = _workload()
    ctx = pslr.from_workload(w)
    ctx.build_lowrank(w["m"], w["rank"])
    lib = pslr.load()
    b = torch.tensor(np.random.default_rng(3).uniform(-1, 1, w["A"].n), device=dev)
    z = torch.zeros_like(b)
    old = ctx.set_wait_limit(0)
    assert _noalloc(lib, ctx, b, z, 0, 0) == pslr.PSLR_OK  # the launch itself succeeds
    assert ctx.sync(check=False) == pslr.PSLR_ERR_TIMEOUT
    ctx.set_wait_limit(old)
    z_ref = torch.zeros_like(b)
    ctx.apply(b, z_ref)
    z_na = torch.full_like(b, float("nan"))
    assert _noalloc(lib, ctx, b, z_na, 0, 0) == pslr.PSLR_OK
    assert ctx.sync(check=False) == pslr.PSLR_OK
    assert np.array_equal(z_na.cpu().numpy(), z_ref.cpu().numpy())
    ctx.close()


def test_apply_noalloc_rejects_too_large(dev):
    """A context whose scratch (3(q+1) + s r values + 256 bytes) exceeds the
    16 MiB array is rejected with PSLR_ERR_TOO_LARGE before anything runs:
    112^3 unknowns cut into 8^3 boxes leave q > 690,000 interface unknowns."""
    from paper_2002_00917_gb300 import pslr

    N = 112
    A = G.shifted_laplacian((N, N, N), 0.01)
    ctx = pslr.Pslr(A, dims=(N, N, N), splits=(14, 14, 14), factor=0)
    q = ctx.info["q"]
    assert 256 + 8 * 3 * (q + 1) > 16 << 20, q
    lib = pslr.load()
    b = torch.zeros(A.n, device=dev, dtype=torch.float64)
    z = torch.zeros_like(b)
    st = _noalloc(lib, ctx, b, z, 0, 0)
    assert st == pslr.PSLR_ERR_TOO_LARGE
    assert "scratch" in lib.pslr_last_error(ctx.h).decode()
    assert ctx.sync(check=False) == pslr.PSLR_OK
    ctx.close()
