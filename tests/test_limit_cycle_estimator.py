"""The limit-cycle estimator (tests/_cycle.py) on series whose period is
known: noisy bursts with a fixed period, a decaying amplitude, and one burst
left out, which the pooled median absorbs."""
import numpy as np

from tests import _cycle as Y


def _bursts(period, n_steps, height, rng, noise=0.3, skip=()):
    t = (np.arange(n_steps // Y.EVERY) + 1) * Y.EVERY
    M = np.ones(t.size)
    for k in range(1, n_steps // period + 1):
        if k in skip:
            continue
        M += height * np.exp(-0.5 * ((t - k * period) / (0.12 * period)) ** 2)
    return M + noise * rng.standard_normal(t.size)


def test_period_and_height_of_regular_bursts():
    rng = np.random.default_rng(0)
    series = [_bursts(1700, Y.STEPS, 3.0, rng) for _ in range(4)]
    period, height, n = Y.ensemble_stats(series)
    assert abs(period - 1700) <= 20 and n >= 4 * 4
    assert abs(height - 4.0) <= 0.2


def test_a_missing_burst_moves_the_median_little():
    rng = np.random.default_rng(1)
    series = [_bursts(1700, Y.STEPS, 3.0, rng, skip=(4,))] + [_bursts(1700, Y.STEPS, 3.0, rng) for _ in range(5)]
    period, _, _ = Y.ensemble_stats(series)
    assert abs(period - 1700) <= 20


def test_different_periods_are_told_apart():
    rng = np.random.default_rng(2)
    p1, _, _ = Y.ensemble_stats([_bursts(1700, Y.STEPS, 3.0, rng) for _ in range(4)])
    p2, _, _ = Y.ensemble_stats([_bursts(1800, Y.STEPS, 3.0, rng) for _ in range(4)])
    assert p2 - p1 >= 60
