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


def _brute_bytes(orc, n, m, r, vs, vb):
    """Pass by pass over the oracle's explicit blocks: each pass streams its
    CSR arrays (values, int32 columns, int32 row pointers; a local solve has an
    L and a U sweep, each with its own row pointers) and reads its input and
    writes its output vector once."""
    def csr_bytes(name, sweeps=1):
        rp, ci, val, shape = orc.block(name)
        return len(val) * vs + len(ci) * 4 + sweeps * 4 * len(rp)

    total = 0
    for _ in range(m + 2):  # B solves (Algorithm 3 steps 2 and 5, and each series term)
        total += csr_bytes("LU_B", 2) + 2 * vs * orc.p
    for _ in range(m + 1):  # C0 solves
        total += csr_bytes("LU_C0", 2) + 2 * vs * orc.q
    for _ in range(m + 1):  # E and F products
        total += csr_bytes("E") + vs * (orc.p + orc.q)
        total += csr_bytes("F") + vs * (orc.q + orc.p)
    for _ in range(m):  # C_g products
        total += csr_bytes("Cg") + vs * 2 * orc.q
    return total + 2 * orc.q * r * vb + 2 * n * vs


@pytest.mark.parametrize("kind,dims,splits", [("lap", (12, 10, 8), (3, 2, 2)), ("cd", (9, 8, 7), (2, 2, 1))])
def test_apply_bytes_by_blocks_counts_every_pass(kind, dims, splits):
    """The closed-form count equals a pass-by-pass sum over the oracle's
    blocks, in both precisions."""
    import bench
    import oracle as O
    from pslr_inputs import configs as C

    w = C.small_problem(kind, dims, splits, factor=0, m=3, rank=5)
    orc = O.from_workload(w)
    for prec, vs, vb in (("fp64", 8, 8), ("fp32", 4, 2)):
        assert bench.bytes_of_oracle(orc, w["A"].n, 3, 5, prec) == _brute_bytes(orc, w["A"].n, 3, 5, vs, vb)


@pytest.mark.parametrize("kind,dims,splits", [("lap", (12, 10, 8), (3, 2, 2)), ("cd", (16, 12, 8), (2, 2, 2))])
def test_gpu_arm_and_reference_arm_count_the_same_bytes(kind, dims, splits):
    """The GPU arm counts from the library's set-up report (pslr_plan, host
    only) and the reference arm from the oracle's blocks: the same number."""
    import bench
    import oracle as O
    from paper_2002_00917_gb300 import build, pslr
    from pslr_inputs import configs as C

    build.build()
    w = C.small_problem(kind, dims, splits, factor=0, m=5, rank=7)
    info = pslr.plan(w["A"], w["dims"], w["splits"], factor=0, m=5, rank=7)[0]
    orc = O.from_workload(w)
    for prec in ("fp64", "fp32"):
        assert bench.bytes_of_info(info, prec) == bench.bytes_of_oracle(orc, w["A"].n, 5, 7, prec)


def test_bf16_round_is_nearest_even():
    """BF16 keeps 8 significant bits: near 1 its spacing is 2^-7."""
    import numpy as np

    import bench

    u = 2.0 ** -7
    x = np.array([1.0, 1.0 + u / 2, 1.0 + 3 * u / 2, 1.0 + 0.75 * u, -(1.0 + 0.25 * u), 1.0 + u / 2 + 2.0 ** -20])
    want = np.array([1.0, 1.0, 1.0 + 2 * u, 1.0 + u, -1.0, 1.0 + u])  # halfway cases go to the even neighbour
    assert np.array_equal(bench.bf16_round(x), want)
