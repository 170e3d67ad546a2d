"""Checkpoint of the low-rank term on the GPU: a term built by the device
Arnoldi, saved, and loaded into a new context set up from the same matrix
gives a bit-identical apply; a context with another reordering refuses it."""
import numpy as np
import pytest

from pslr_inputs import configs as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_lowrank_checkpoint_round_trip(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build, pslr

    build.build()
    w = C.small_problem("lap", (13, 11, 9), (3, 2, 2), m=3, rank=6, K=3)
    a = pslr.from_workload(w)
    a.build_lowrank(3, 6)
    path = tmp_path / "lowrank.npz"
    a.save_lowrank(path)
    b = pslr.from_workload(w)
    assert b.load_lowrank(path) == a.info["rank"]
    x = torch.tensor(np.random.default_rng(5).uniform(-1, 1, w["A"].n), device="cuda")
    za, zb = torch.empty_like(x), torch.empty_like(x)
    a.apply(x, za)
    b.apply(x, zb)
    a.sync()
    b.sync()
    assert torch.equal(za, zb)
    other = pslr.Pslr(w["A"], dims=w["dims"], splits=(2, 2, 2), factor=w["factor"])
    with pytest.raises(ValueError):
        other.load_lowrank(path)
