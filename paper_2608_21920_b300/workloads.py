"""Synthetic workloads of the method (all seeded; the paper uses no dataset)
and a runner that records their diagnostic traces.

* production: one gap, Nx = 16384, dx = 0.05, 64 cold electrons per cell,
  alpha = 1.5, b = 0.1, rho_c = 1e7 cm, cap 1e8 (leptons + photons) with the
  weight-conserving merge;
* batch: 256 independent gaps with Nx ~ U[1024, 8192], alpha ~ U[-1, 3],
  b ~ logU[0.03, 0.3], rho_c ~ logU[1e6, 1e8] cm, 8-64 electrons per cell,
  per-gap seeds 0..255, per-gap cap 16x the initial count; each gap's row is
  drawn from Philox keyed by (gap index, table channel), so the table is
  reproducible gap by gap.

QED scales (Sect. 6.1 rescaling): physical scales put no pairs inside these
boxes, so lambda_hat = lambda_C / d_e = 1e-5 and rate multiplier 2 are used
throughout, and the curvature radius maps to rho_hat = 20 rho_c / (1e7 cm)
(20 d_e at the fiducial 1e7 cm).

    python -m paper_2608_21920_b300.workloads production --steps 200000 --every 200 --out traces.npz
    python -m paper_2608_21920_b300.workloads batch --steps 20000 --every 100 --out batch.npz
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

BC_SURFACE, INIT_COLD = 0, 1
LAMBDA_HAT, RATE_MULT, RHO_HAT_AT_1E7 = 1e-5, 2.0, 20.0
TABLE_CHANNEL = 11  # Philox key word of the batch parameter table


def rho_hat(rho_c_cm: float) -> float:
    return RHO_HAT_AT_1E7 * rho_c_cm / 1e7


def production(precision: str = "fp32", seed: int = 0) -> dict:
    """The production single gap (dt = 0.45 dx)."""
    return dict(nx=16384, dx=0.05, dt=0.0225, ppc=64, density=1.0, alpha=1.5, b=0.1,
                lambda_hat=LAMBDA_HAT, rho_hat=rho_hat(1e7), rate_mult=RATE_MULT, qed=1,
                init=INIT_COLD, boundary=BC_SURFACE, cap=100_000_000, seed=seed, gap_index=0)


def batch_row(i: int) -> dict:
    """Parameters of gap i of the batch, from Philox keyed by (i, table channel)."""
    rng = np.random.Generator(np.random.Philox(key=np.array([i, TABLE_CHANNEL], dtype=np.uint64)))
    nx = int(rng.integers(1024, 8193))
    alpha = float(rng.uniform(-1.0, 3.0))
    b = float(math.exp(rng.uniform(math.log(0.03), math.log(0.3))))
    rho_c = float(math.exp(rng.uniform(math.log(1e6), math.log(1e8))))
    ppc = int(rng.integers(8, 65))
    return dict(nx=nx, dx=0.1, dt=0.045, ppc=ppc, density=1.0, alpha=alpha, b=b,
                lambda_hat=LAMBDA_HAT, rho_hat=rho_hat(rho_c), rate_mult=RATE_MULT, qed=1,
                init=INIT_COLD, boundary=BC_SURFACE, cap=16 * nx * ppc, seed=i, gap_index=i)


def batch(n_gaps: int = 256) -> list[dict]:
    return [batch_row(i) for i in range(n_gaps)]


# Concurrency-model scan (App. B empirical fit): 36 parameter sets in five
# one-at-a-time sweeps around the Fig. 2 point (alpha = 2, t_x = t_pm = 1e-3,
# t_acc = 4e-8, g3 = 8e-8, units of t_esc).  The paper names the sweeps and
# the count but not their ranges; these span a factor 10 either way in g3
# and t_acc, about 3 in t_x and t_pm, and alpha in [1.25, 4].
SCAN_BASE = dict(alpha=2.0, t_x=1e-3, t_pm=1e-3, t_acc=4e-8, g3=8e-8)


def concurrency_scan() -> list[dict]:
    """The 36 sets, each with the name of its sweep."""
    out = []
    sweeps = (("g3", np.geomspace(8e-9, 8e-7, 8)), ("t_pm", np.geomspace(3e-4, 3e-3, 7)),
              ("t_x", np.geomspace(3e-4, 3e-3, 7)), ("t_acc", np.geomspace(4e-9, 4e-7, 7)),
              ("alpha", np.linspace(1.25, 4.0, 7)))
    for name, values in sweeps:
        for v in values:
            out.append(dict(SCAN_BASE, **{name: float(v)}, sweep=name))
    return out


TRACE_KEYS = ("M_avg", "M_peak", "E_min", "E_max", "E_abs_max", "n_electrons", "n_positrons", "n_photons")


def run_traces(params, steps: int, every: int, precision: str = "fp32", graph_chunk: int = 0,
               spectrum_gap: int | None = 0, tile: int = 0, threads: int = 0, rebin_every: int = 0,
               log=None) -> dict:
    """Advance the gaps for `steps` steps and sample every `every` steps the
    per-gap diagnostics (TRACE_KEYS, counters, and the |E_k|^2 spectrum of
    one gap).  Returns numpy arrays: trace[key] of shape [samples, gaps]."""
    import torch

    from .gap import Gap

    plist = [params] if isinstance(params, dict) else list(params)
    t_init = time.perf_counter()
    g = Gap(plist, precision=precision, tile=tile, threads=threads, rebin_every=rebin_every)
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t_init
    n = len(plist)
    S = steps // every
    tr = {k: np.zeros((S + 1, n)) for k in TRACE_KEYS}
    tr["pairs"] = np.zeros((S + 1, n))
    tr["merged"] = np.zeros((S + 1, n))
    spectra = []
    step_ms = []

    def sample(j):
        for i in range(n):
            d = g.diag(i, spectrum=(spectrum_gap == i))
            for k in TRACE_KEYS:
                tr[k][j, i] = d[k]
            tr["pairs"][j, i] = d["counters"]["pairs"]
            tr["merged"][j, i] = d["counters"]["merged"]
            if spectrum_gap == i:
                spectra.append(d["spectrum"])

    sample(0)
    s = torch.cuda.Stream() if graph_chunk > 0 else torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for j in range(1, S + 1):
        with torch.cuda.stream(s):
            e0.record(s)
            g.step(every, graph_chunk=graph_chunk if graph_chunk and every % graph_chunk == 0 else 0)
            e1.record(s)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1) / every)
        sample(j)
        if log and j % max(1, S // 20) == 0:
            nl = tr["n_electrons"][j].sum() + tr["n_positrons"][j].sum()
            log(f"step {j * every}: leptons {nl:.3g}, photons {tr['n_photons'][j].sum():.3g}, "
                f"{step_ms[-1]:.3f} ms/step")
    out = {k: v for k, v in tr.items()}
    out["step"] = np.arange(S + 1) * every
    out["ms_per_step"] = np.array(step_ms)
    out["t_init_s"] = np.array(t_init)
    if spectra:
        out["spectrum"] = np.array(spectra)
    for k in ("alpha", "b", "rho_hat", "nx", "ppc", "dx", "dt", "cap", "gap_length"):
        out["param_" + k] = np.array([p.get(k, 0) for p in plist], dtype=float)
    g.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["production", "batch"])
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--gaps", type=int, default=256)
    ap.add_argument("--graph-chunk", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--rebin-every", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    params = production(a.precision) if a.workload == "production" else batch(a.gaps)
    t0 = time.perf_counter()
    tr = run_traces(params, a.steps, a.every, a.precision, graph_chunk=a.graph_chunk,
                    spectrum_gap=0, tile=a.tile, threads=a.threads, rebin_every=a.rebin_every,
                    log=lambda m: print(m, flush=True))
    wall = time.perf_counter() - t0
    np.savez_compressed(a.out, **tr)
    nl = tr["n_electrons"] + tr["n_positrons"]
    summary = dict(workload=a.workload, precision=a.precision, steps=a.steps, wall_s=wall,
                   init_s=float(tr["t_init_s"]), ms_per_step_median=float(np.median(tr["ms_per_step"])),
                   lepton_steps_per_s=float(np.mean(nl[1:].sum(axis=1)) / (np.median(tr["ms_per_step"]) / 1e3)),
                   leptons_final=float(nl[-1].sum()), photons_final=float(tr["n_photons"][-1].sum()),
                   pairs=float(tr["pairs"][-1].sum()), merged=float(tr["merged"][-1].sum()))
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
