"""The Section 4.1 study driver in its GPU-free mode (host set-up only), and
its fill factors against the ones Tables 1 and 3 print for the same 50^3
problem with ILUT(1e-2).  The geometric split stands in for METIS, so the
comparison allows a few percent; it checks the ILUT reading (drop tolerance
relative to the row's mean modulus) and the fill-factor definitions of
Section 4."""
import pytest


@pytest.fixture(scope="module")
def ex():
    from paper_2002_00917_gb300 import build, experiments

    build.build()
    return experiments


def test_s_sweep_fill_factors_follow_table1(ex, capsys):
    recs = ex.main(["s", "--dry-run"])
    assert [r["s"] for r in recs] == [8, 16, 27, 36, 45, 54]
    # Table 1 (s = 5, 15, 25, 35, 45, 55): fill (ILU) and fill (low-rank)
    ilu = [2.68, 2.45, 2.30, 2.23, 2.17, 2.11]
    lr = [.19, .37, .49, .55, .60, .66]
    for rec, fi, fl in zip(recs, ilu, lr):
        assert abs(rec["fill_ilu"] - fi) <= 0.05 * fi, (rec, fi)
        if rec["s"] >= 27:  # the interface size of s = 5 and 15 differs from METIS's most
            assert abs(rec["fill_lr"] - fl) <= 0.08 * fl, (rec, fl)
    ilus = [r["fill_ilu"] for r in recs]
    lrs = [r["fill_lr"] for r in recs]
    assert ilus == sorted(ilus, reverse=True) and lrs == sorted(lrs)  # the trends Table 1 shows
    assert len(capsys.readouterr().out.strip().splitlines()) == 6


def test_rank_sweep_low_rank_fill_follows_table3(ex):
    recs = ex.main(["rank", "--dry-run"])
    assert [r["r"] for r in recs] == [0, 15, 30, 45, 60, 75]
    for rec, fl in zip(recs, [0.0, .55, 1.10, 1.65, 2.20, 2.75]):  # Table 3, fill (low-rank)
        assert abs(rec["fill_lr"] - fl) <= 0.02 * max(fl, 1e-9), (rec, fl)
        assert abs(rec["fill_ilu"] - 2.24) <= 0.03 * 2.24  # Table 3, fill (ILU)
        assert rec["levels_B"] == recs[0]["levels_B"]


def test_m_sweep_runs_are_the_table2_set(ex):
    assert [(s, sp, m, r) for s, sp, m, r in ex.runs("m")] == [(0.05, (3, 3, 4), m, 15) for m in range(6)]
    assert ex.runs("rank", 0.14)[0][0] == 0.14
    with pytest.raises(ValueError):
        ex.runs("threads")


def test_lap_sweep_total_fill_follows_table6(ex):
    """Table 6 prints the total fill (ILU + low-rank) of PSLR with s = 35,
    m = 3, r = 15: 2.76 (32^3, shift .16) and 2.85 (64^3, shift .08).  The
    3x3x4 split gives the same within 3%.  128^3 runs 256 parts instead of
    35 (the paper's 3.15 is not comparable) and is checked for a sound
    layout only."""
    recs = ex.main(["lap", "--dry-run"])
    assert [r["dims"][0] for r in recs] == [32, 64, 128]
    for rec, ft in zip(recs[:2], (2.76, 2.85)):
        assert abs(rec["fill_total"] - ft) <= 0.03 * ft, (rec, ft)
        assert abs(rec["fill_total"] - rec["fill_ilu"] - rec["fill_lr"]) < 1e-3
    assert recs[2]["s"] == 256
