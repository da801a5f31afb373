"""Parameter scan of the discharge concurrency model (App. B, empirical
fitting formula eq. Mpm_empirical): the ODE solutions of many parameter sets
integrated together by the batched RK4 kernel (hard gate, FP64), their peak
multiplicities, and log-space least-squares fits of those peaks.

Per set: step dt = min(2e-4, 0.2 min(t_x, t_pm)) t_esc (the ignition grows
on the scale t_pm, the gate on t_x); every set takes the same number of
steps, enough for the smallest dt to reach `t_end`.  Peaks are the local
maxima of m_pm above 100 in the trace sampled every `every` steps; the first
discharge (loading from the initial state) is left out of the mean.

    python -m paper_2608_21920_b300.scan [--t-end 30] [--every 5]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

PEAK_FLOOR = 100.0


def step_sizes(sets) -> np.ndarray:
    return np.array([min(2e-4, 0.2 * min(q["t_x"], q["t_pm"])) for q in sets])


def peak_indices(m: np.ndarray) -> np.ndarray:
    """Local maxima m[i-1] < m[i] >= m[i+1] above PEAK_FLOOR."""
    i = np.where((m[1:-1] > m[:-2]) & (m[1:-1] >= m[2:]))[0] + 1
    return i[m[i] > PEAK_FLOOR]


def fit(sets, peak_mean) -> dict:
    """Log-space least squares of the peak multiplicity:
    * compound: ln M = ln C + a ln(t_acc/(t_x g3)) + b ln alpha;
    * free: one exponent per parameter (t_acc, g3, t_x, t_pm, alpha);
    * the paper's exponents (1, 1/4) with C alone, and the ratio of every
      set to 11 (t_acc/(t_x g3)) alpha^(1/4)."""
    M = np.asarray(peak_mean, dtype=float)
    X = np.array([q["t_acc"] / (q["t_x"] * q["g3"]) for q in sets])
    al = np.array([q["alpha"] for q in sets])
    y = np.log(M)
    A = np.stack([np.ones_like(X), np.log(X), np.log(al)], axis=1)
    c, *_ = np.linalg.lstsq(A, y, rcond=None)
    keys = ("t_acc", "g3", "t_x", "t_pm", "alpha")
    A2 = np.stack([np.ones_like(X)] + [np.log([q[k] for q in sets]) for k in keys], axis=1)
    c2, *_ = np.linalg.lstsq(A2, y, rcond=None)
    C_paper_exponents = float(np.exp(np.mean(y - np.log(X * al ** 0.25))))
    ratio = M / (11.0 * X * al ** 0.25)
    return {"C": float(np.exp(c[0])), "a": float(c[1]), "b": float(c[2]),
            "free": {"C": float(np.exp(c2[0])), **{k: float(v) for k, v in zip(keys, c2[1:])}},
            "C_paper_exponents": C_paper_exponents,
            "ratio_to_paper": ratio.tolist(),
            "max_rel_dev_paper": float(np.max(np.abs(ratio - 1.0)))}


def run(sets=None, t_end: float = 30.0, every: int = 5, device: str = "cuda") -> dict:
    """Integrate the sets on the GPU and return per-set peaks and the fits."""
    import torch

    from . import ode, workloads
    if sets is None:
        sets = workloads.concurrency_scan()
    dt = step_sizes(sets)
    nsteps = int(math.ceil(t_end / dt.min()))
    nsteps -= nsteps % every
    dev = torch.device(device)
    p = torch.tensor([[q["alpha"], q["t_x"], q["t_pm"], q["t_acc"], q["g3"]] for q in sets],
                     dtype=torch.float64, device=dev)
    y0 = torch.tensor([[1.0, 0.0, 1.0, 0.0]] * len(sets), dtype=torch.float64, device=dev)
    dtt = torch.tensor(dt, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out, _ = ode.forward(p, y0, dtt, nsteps, every=every)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    m = out[:, :, 0].cpu().numpy()
    n_peaks, peak_mean, first_peak = [], [], []
    for b in range(len(sets)):
        i = peak_indices(m[:, b])
        n_peaks.append(int(i.size))
        first_peak.append(float(m[i[0], b]) if i.size else float("nan"))
        peak_mean.append(float(m[i[1:], b].mean()) if i.size > 1 else float("nan"))
    res = {"sets": sets, "dt": dt.tolist(), "nsteps": nsteps, "every": every, "ms": ms,
           "rk4_steps_per_s": len(sets) * nsteps / (ms / 1e3),
           "n_peaks": n_peaks, "first_peak": first_peak, "peak_mean": peak_mean}
    if all(np.isfinite(peak_mean)):
        res["fit"] = fit(sets, peak_mean)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--t-end", type=float, default=30.0)
    ap.add_argument("--every", type=int, default=5)
    a = ap.parse_args()
    r = run(t_end=a.t_end, every=a.every)
    f = r.get("fit", {})
    print(json.dumps({"sets": len(r["sets"]), "nsteps": r["nsteps"], "ms": r["ms"],
                      "rk4_steps_per_s": r["rk4_steps_per_s"], "n_peaks_min": min(r["n_peaks"]),
                      "fit": {k: v for k, v in f.items() if k != "ratio_to_paper"}}), flush=True)


if __name__ == "__main__":
    main()
