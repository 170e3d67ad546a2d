"""pslr_apply_noalloc: the apply for callers that cannot allocate device memory
when they apply the preconditioner (their device memory belongs to a pool
allocator of their own and cudaMalloc/cudaFree are off limits).  It runs the
apply kernel on a scratch array that lives inside the library instead of on
buffers the context allocated, so its result must equal pslr_apply's.  This
file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from pslr_inputs import configs as Cf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "fp32"])
def test_apply_noalloc_matches_apply_twice(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build, pslr

    build.build()
    w = Cf.small_problem("cd", (12, 10, 8), (3, 2, 2), factor=0, m=3, rank=6, K=3)
    ctx = pslr.from_workload(w)
    ctx.build_lowrank(w["m"], w["rank"])
    lib = pslr.load()
    dt = torch.float64 if prec == 0 else torch.float32
    stream = pslr._stream(None)
    rng = np.random.default_rng(11)
    for transpose in (0, 1):
        for call in range(2):  # two calls in a row: the shared scratch keeps old contents
            b = torch.tensor(rng.uniform(-1, 1, w["A"].n), device="cuda", dtype=dt)
            z_ref = torch.zeros_like(b)
            z_na = torch.full_like(b, float("nan"))
            ctx.apply(b, z_ref, transpose=bool(transpose))
            st = lib.pslr_apply_noalloc(ctx.h, C.c_void_p(b.data_ptr()), C.c_void_p(z_na.data_ptr()),
                                        prec, transpose, stream)
            assert st == pslr.PSLR_OK, lib.pslr_last_error(ctx.h).decode()
            ctx.sync()
            rel = _rel(z_na.cpu().double().numpy(), z_ref.cpu().double().numpy())
            assert rel <= tol, (transpose, call, rel)
