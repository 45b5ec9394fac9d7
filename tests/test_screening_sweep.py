"""Screening sweep (paper_2412_11081_gb300/screening_sweep.py): the option
families on the CPU, and a short sweep on the GPU whose kept-item counts
fall and errors rise with the thresholds."""
import pytest

from paper_2412_11081_gb300 import screening_sweep as ss


def test_threshold_families():
    assert ss._thetas("reference", 1.0, 1e-10) == {k: 0.0 for k in ("C", "dC", "V", "dV", "D", "CS")}
    th = ss._thetas("C+dC", 1e-6, 1e-10)
    assert th["C"] == th["dC"] == 1e-6 and th["V"] == th["dV"] == th["D"] == th["CS"] == 0.0
    th = ss._thetas("V+dV", 1e-6, 1e-10)
    assert th["V"] == th["dV"] == 1e-6 and th["C"] == th["D"] == th["CS"] == 0.0
    th = ss._thetas("D", 1e-4, 1e-10)
    assert th["D"] == 1e-4 and sum(v for k, v in th.items() if k != "D") == 0.0
    th = ss._thetas("CS+pre", 1e-6, 1e-10)
    assert th["CS"] == 1e-6 and all(th[k] == 1e-10 for k in ("C", "dC", "V", "dV", "D"))
    with pytest.raises(ValueError):
        ss._thetas("X", 1.0, 0.0)


@pytest.mark.gpu
def test_sweep_on_diamond8():
    from paper_2412_11081_gb300 import inputs
    w = inputs.diamond8()
    rows = ss.sweep(w, [1e-10, 1e-4, 1e-1], families=("CS", "D"), reps=1, split=True)
    ref = rows[0]
    assert ref["family"] == "reference" and ref["errF"] == 0.0
    for fam in ("CS", "D"):
        r = [x for x in rows if x["family"] == fam]
        trip = [x["triplets"] for x in r]
        assert trip == sorted(trip, reverse=True) and trip[0] <= ref["triplets"]
        assert r[0]["errF"] < 1e-8 and r[0]["errS"] < 1e-8   # 1e-10 changes almost nothing
        assert r[-1]["triplets"] < ref["triplets"]            # 0.1 drops items
        assert all(x["ms_fp64"] > 0 and x["ms_bf16x6"] > 0 for x in r)
