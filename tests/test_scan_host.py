"""Host logic of the concurrency-model scan (no GPU): the 36 sets, the step
rule, peak picking and the log-space fits on synthetic peaks."""
import numpy as np
import pytest

from paper_2608_21920_b300 import scan, workloads


def test_scan_sets_are_five_sweeps_around_fig2():
    sets = workloads.concurrency_scan()
    assert len(sets) == 36
    names = [q["sweep"] for q in sets]
    assert [names.count(k) for k in ("g3", "t_pm", "t_x", "t_acc", "alpha")] == [8, 7, 7, 7, 7]
    for q in sets:  # one parameter off the Fig. 2 point at a time
        off = [k for k in workloads.SCAN_BASE if q[k] != workloads.SCAN_BASE[k]]
        assert off in ([], [q["sweep"]])


def test_step_rule():
    dt = scan.step_sizes([dict(t_x=1e-3, t_pm=1e-3), dict(t_x=3e-4, t_pm=1e-3), dict(t_x=1e-3, t_pm=5e-4)])
    assert np.allclose(dt, [2e-4, 6e-5, 1e-4])


def test_peak_indices():
    m = np.array([0, 50, 150, 120, 130, 130, 90, 400, 10.0])
    assert list(scan.peak_indices(m)) == [2, 4, 7]


def test_fit_recovers_exact_power_law():
    sets = workloads.concurrency_scan()
    X = np.array([q["t_acc"] / (q["t_x"] * q["g3"]) for q in sets])
    al = np.array([q["alpha"] for q in sets])
    f = scan.fit(sets, 11.0 * X * al ** 0.25)
    assert f["C"] == pytest.approx(11.0, rel=1e-10)
    assert f["a"] == pytest.approx(1.0, abs=1e-10) and f["b"] == pytest.approx(0.25, abs=1e-10)
    fr = f["free"]
    assert fr["t_acc"] == pytest.approx(1.0, abs=1e-9) and fr["g3"] == pytest.approx(-1.0, abs=1e-9)
    assert fr["t_x"] == pytest.approx(-1.0, abs=1e-9) and abs(fr["t_pm"]) < 1e-9
    assert f["max_rel_dev_paper"] < 1e-12 and f["C_paper_exponents"] == pytest.approx(11.0, rel=1e-12)
