"""One run of the Section 4.1 study driver on the GPU: 50^3, shift .05,
3x3x4 split, ILUT(1e-2), m = 3, r = 15 (the paper's Table 1 row s = 35 and
Table 3 row r = 15 print 83 and 86 iterations).  FGMRES converges, the host
dry run and the device context agree on the layout figures, and the count
stays in the range those tables print."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_experiment_run_on_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00917_gb300 import build, experiments
    from pslr_inputs import generators as G

    build.build()
    A = G.shifted_laplacian(experiments.DIMS, 0.05)
    dry = experiments.one(A, 0.05, (3, 3, 4), 3, 15, dry_run=True)
    rec = experiments.one(A, 0.05, (3, 3, 4), 3, 15)
    assert rec["converged"] and rec["relres"] <= 1e-8
    for k in ("q", "fill_ilu", "fill_lr", "levels_B", "levels_C0"):
        assert rec[k] == dry[k], k
    assert 70 <= rec["its"] <= 110, rec
