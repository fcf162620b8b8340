"""The caloric-curve analysis of the glass quench on curves of known shape (no GPU), and a
short quench through the library (GPU)."""
import numpy as np
import pytest

from paper_1105_5613_gb300 import glass_quench as gq


def test_analysis_recovers_a_known_break():
    T = np.linspace(3.0, 0.001, 3000)
    a, b, Tg = -2.0, 1.5, 0.2
    liquid = a + b * T ** 0.6
    slope = 0.6 * b * Tg ** -0.4 * 0.35           # glass branch: a smaller slope
    glass = a + b * Tg ** 0.6 + slope * (T - Tg)
    U = np.where(T >= Tg, liquid, glass)
    res = gq.analyse(T, U, liquid_min=0.5, glass_max=0.1)
    assert res["liquid_fit"]["a"] == pytest.approx(a, abs=1e-9)
    assert res["liquid_fit"]["b"] == pytest.approx(b, abs=1e-9)
    assert res["glass_fit"]["d"] == pytest.approx(slope, rel=1e-9)
    # the straight glass line meets the liquid curve at Tg (tangent-like crossing below it)
    assert abs(res["T_g"] - Tg) < 0.05


def test_analysis_without_a_break_reports_none():
    T = np.linspace(3.0, 0.001, 500)
    U = -2.0 + 1.5 * T ** 0.6
    res = gq.analyse(T, U, liquid_min=0.5, glass_max=0.1)
    assert np.isnan(res["T_g"]) or res["T_g"] < 0.12


@pytest.mark.gpu
def test_short_quench_runs_through_the_library():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    res = gq.run(ncell=12, heat_steps=2000, cool_steps=20000, every=500, gr_bins=100)
    c = res["curve"]
    T, U = np.array(c["T"]), np.array(c["U"])
    assert np.all(np.isfinite(U)) and len(U) == 2000 // 500 + 20000 // 500
    # cooling lowers the potential energy; the thermostat follows the ramp
    assert U[-1] < U[3] - 0.5
    assert T[-1] < 0.1 and 2.0 < np.mean(T[:4]) < 4.5
    g = np.array(res["gr"]["total"])
    r = np.array(res["gr"]["r"])
    assert 0.8 < r[np.argmax(g)] < 1.2  # first peak near one particle diameter (Sec. 4)
