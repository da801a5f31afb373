"""Limit-cycle statistics of a PIC discharge, shared by the CPU test of the
estimator and the GPU-against-oracle test.

The paper's PIC discharge repeats in bursts (Sect. 6.2; the concurrency
model's cycle is Sect. 5.4's t_cycle).  Its period is read as the interval
between successive maxima of the gap-peak multiplicity M_peak(t), the first
discharge left out.  M_peak is noisy from step to step, so a maximum is a
burst maximum of the series smoothed over 200 steps whose prominence is at
least a quarter of the smoothed series' range after the first discharge
started (step 500); an ensemble of seeds pools its intervals, and the period
is their median (robust to a burst too weak to count, which doubles one
interval), the peak multiplicity the mean smoothed M_peak at the maxima."""
import numpy as np
from scipy.signal import find_peaks

STEPS, EVERY, T_START, SMOOTH_STEPS = 12000, 10, 500, 200


def burst_maxima(M, every=EVERY, t_start=T_START, smooth_steps=SMOOTH_STEPS):
    """Steps and smoothed heights of the burst maxima of a series sampled
    every `every` steps (sample i at step (i + 1) every)."""
    M = np.asarray(M, dtype=float)
    w = max(1, smooth_steps // every)
    s = np.convolve(M, np.ones(w) / w, mode="same")
    t = (np.arange(M.size) + 1) * every
    sel = t >= t_start
    pk, _ = find_peaks(s, prominence=0.25 * (s[sel].max() - s[sel].min()))
    pk = pk[t[pk] >= t_start]
    return t[pk], s[pk]


def ensemble_stats(series, every=EVERY):
    """(period in steps, mean peak multiplicity, intervals pooled) of an
    ensemble of M_peak series, each with its first discharge left out."""
    d, h = [], []
    for M in series:
        tp, hp = burst_maxima(M, every)
        d.extend(np.diff(tp)[1:])
        h.extend(hp[1:])
    return float(np.median(d)), float(np.mean(h)), len(d)


def oracle_mpeak_series(cfg):
    """M_peak every EVERY steps over STEPS steps of the oracle (one process)."""
    import oracle as O
    o = O.Sim(**{k: v for k, v in cfg.items() if k in O.DEFAULTS})
    out = []
    for _ in range(STEPS // EVERY):
        o.step(EVERY)
        out.append(o.diag()["M_peak"])
    return np.array(out)
