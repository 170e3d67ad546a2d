import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)


def dense_lu_product(o, name):
    """B~ = L U (or C0~) from an oracle's exported ILU(0) factor: the matrix whose
    inverse the method applies when it writes B^{-1} (Algorithm 1, steps 3-4)."""
    D = o.dense_block(name)
    L = np.tril(D, -1) + np.eye(D.shape[0])
    U = np.triu(D)
    return L @ U


def dense_operators(o, factor):
    """Dense B~, E, F, C, C0~, C_g of an oracle set-up (reordered numbering)."""
    B = o.dense_block("B")
    E = o.dense_block("E")
    F = o.dense_block("F")
    Cc = o.dense_block("C")
    C0 = o.dense_block("C0")
    Cg = o.dense_block("Cg")
    if factor == 0:
        Bt = dense_lu_product(o, "LU_B")
        C0t = dense_lu_product(o, "LU_C0")
    else:
        Bt, C0t = B, C0
    return dict(B=B, Bt=Bt, E=E, F=F, C=Cc, C0=C0, C0t=C0t, Cg=Cg)
