"""Host-side accounting of bench.py (no GPU): the FP64 work it attributes to
the Krylov part of an FGMRES run."""
import pytest

pytest.importorskip("torch")


def test_krylov_work_counts_cgs2_spmv_and_normalisation():
    """FGMRES(restart) with k basis vectors in a step does 4 k n FMAs of CGS2
    (two projections and two updates), nnz for A z and n for the
    normalisation; a restart resets k to 1."""
    import bench

    n, nnz = 10, 37
    e = bench.krylov_estimate(iters=7, restart=3, n=n, nnz=nnz, ms=5.0, apply_ms=0.5)
    ks = [1, 2, 3, 1, 2, 3, 1]
    assert e["fp64_fma"] == sum(4 * k * n + nnz + n for k in ks)
    assert e["ms_est"] == pytest.approx(5.0 - 7 * 0.5)
    assert e["tflops_est"] == pytest.approx(2.0 * e["fp64_fma"] / (e["ms_est"] * 1e-3) / 1e12)
    assert e["frac_of_fp64_nominal"] == pytest.approx(e["tflops_est"] / e["fp64_nominal_tflops"])


def test_krylov_time_never_negative():
    import bench

    e = bench.krylov_estimate(iters=3, restart=5, n=4, nnz=4, ms=1.0, apply_ms=1.0)
    assert e["ms_est"] > 0.0
