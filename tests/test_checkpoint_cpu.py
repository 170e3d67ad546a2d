"""Checkpoint of the low-rank term (save_lowrank / load_lowrank) on the CPU:
the binding's file logic, with a stand-in for the device context (no GPU).
The GPU path is in tests/test_gpu_checkpoint.py."""
import numpy as np
import pytest

from pslr_inputs import generators as G


class _Stub:
    """The parts of a context the checkpoint uses, on host arrays."""

    def __init__(self, pslr, A, factor=0, drop_tol=0.0, shift_perm=0):
        self.cls = pslr.Pslr
        self._rp, self._ci, self._av = A.rowptr, A.col, A.val
        self.factor, self.drop_tol = factor, drop_tol
        n = A.n
        self._maps = (np.zeros(n, np.int32), np.zeros(n, np.int32), np.roll(np.arange(n, dtype=np.int32), shift_perm))
        self.info = {"m": 0, "rank": 0, "q": 7}
        self.installed = None

    def get_maps(self):
        return self._maps

    def get_lowrank(self):
        r = self.info["rank"]
        rng = np.random.default_rng(r)
        return rng.random((7, r)), rng.random((r, r)), rng.random((r, r))

    def set_lowrank(self, m, V=None, G=None, stream=None):
        self.installed = (m, V, G)

    def __getattr__(self, name):  # the binding's methods, bound to the stub
        return getattr(self.cls, name).__get__(self)


def test_save_and_load_round_trip(tmp_path):
    from paper_2002_00917_gb300 import pslr

    A = G.shifted_laplacian((6, 5), 0.1)
    src = _Stub(pslr, A)
    src.info.update(m=3, rank=4)
    path = tmp_path / "lr.npz"
    src.save_lowrank(path)
    V, H, Gm = src.get_lowrank()
    dst = _Stub(pslr, A)
    assert dst.load_lowrank(path) == 4
    m, V2, G2 = dst.installed
    assert m == 3 and np.array_equal(V2, V) and np.array_equal(G2, Gm)


def test_rank_zero_term_and_mismatches(tmp_path):
    from paper_2002_00917_gb300 import pslr

    A = G.shifted_laplacian((6, 5), 0.1)
    src = _Stub(pslr, A)
    src.info.update(m=2, rank=0)
    path = tmp_path / "lr0.npz"
    src.save_lowrank(path)
    dst = _Stub(pslr, A)
    assert dst.load_lowrank(path) == 0 and dst.installed == (2, None, None)
    B = G.shifted_laplacian((6, 5), 0.2)  # other values
    for other in (_Stub(pslr, B), _Stub(pslr, A, factor=2, drop_tol=1e-2), _Stub(pslr, A, shift_perm=1)):
        with pytest.raises(ValueError):
            other.load_lowrank(path)
