"""Fit of the discharge concurrency model (Sect. 5.2, eq. dis1-dis4) to the
E(t) and pair-multiplicity traces of a batch of PIC gaps, with gradients from
the hand-written discrete adjoint of the batched RK4 integrator (ode.py).

Units.  The model's time unit is t_esc = H_gap / c (H_gap = gap_length, by
default 0.8 Nx dx); its multiplicity m_pm is compared with the PIC's
gap-averaged multiplicity M_avg, and its field eps with the largest |E| over
the gap divided by a scale E_s: the model's unit field (|eps| = 1 switches
photon production on) has no fixed value in PIC units, so ln E_s is fitted
beside ln t_x, ln t_pm, ln t_acc, ln g3.  alpha is the gap's imposed current.
Each gap gets `starts` parameter sets drawn log-uniformly over t_x, t_pm in
[1e-4, 1e-2], t_acc in [1e-8, 1e-7], g3 in [1e-8, 1e-6] (Fig. 2 neighbourhood);
all sets are fitted together by Adam on the log-parameters.

Loss of a set (mean over the trace samples):
    (ln(1 + m) - ln(1 + M))^2 + (|eps| E_s - |E|max)^2 / mean(|E|max^2)
The gate is the smoothed one (H_delta, delta = 1e-2) so that the loss is
differentiable; the PIC itself is not differentiated.

    python -m paper_2608_21920_b300.fit --traces batch.npz --starts 16 --iters 40
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import ode

DELTA = 1e-2
BOUNDS = ((1e-4, 1e-2), (1e-4, 1e-2), (1e-8, 1e-7), (1e-8, 1e-6))  # t_x, t_pm, t_acc, g3


def load_traces(path: str) -> dict:
    z = np.load(path)
    nx, dx, dt = z["param_nx"], z["param_dx"], z["param_dt"]
    steps = z["step"]
    # the model's time unit is the escape time over the gap, H_gap / c
    # (Sect. 5.2); a gap saved with H_gap = 0 had the default 0.8 nx dx
    H = z["param_gap_length"] if "param_gap_length" in z.files else np.zeros_like(nx)
    t_esc = np.where(H > 0, H, 0.8 * nx * dx)
    return dict(M=z["M_avg"], E=z["E_abs_max"], alpha=z["param_alpha"], t_esc=t_esc,
                sample_dt=(steps[1] - steps[0]) * dt)


class Problem:
    """The batched fit: B = gaps x starts parameter sets."""

    def __init__(self, tr: dict, starts: int = 16, every: int = 50, seed: int = 0,
                 dtype=torch.float64, device="cuda"):
        M = torch.as_tensor(tr["M"], dtype=dtype)
        E = torch.as_tensor(tr["E"], dtype=dtype)
        S1, G = M.shape
        self.G, self.starts, self.every = G, starts, every
        self.nsteps = (S1 - 1) * every
        self.B = G * starts
        gi = torch.arange(self.B) // starts
        self.gi = gi
        self.M = M[:, gi].to(device)                       # [T, B]
        self.E = E[:, gi].to(device)
        self.E2 = (self.E ** 2).mean(dim=0).clamp_min(1e-30)
        alpha = torch.as_tensor(tr["alpha"], dtype=dtype)[gi]
        t_esc = torch.as_tensor(tr["t_esc"], dtype=dtype)[gi]
        self.dt = (torch.as_tensor(tr["sample_dt"], dtype=dtype)[gi] / t_esc / every).to(device)
        self.alpha = alpha.to(device)
        g = torch.Generator().manual_seed(seed)
        lo = torch.tensor([math.log(b[0]) for b in BOUNDS], dtype=dtype)
        hi = torch.tensor([math.log(b[1]) for b in BOUNDS], dtype=dtype)
        th = lo + (hi - lo) * torch.rand(self.B, 4, generator=g, dtype=dtype)
        Emax = self.E.max(dim=0).values.cpu().clamp_min(1e-12)
        lnEs = torch.log(Emax / 2.0) + 0.5 * torch.randn(self.B, generator=g, dtype=dtype)
        self.theta = torch.cat([th, lnEs[:, None]], dim=1).to(device).requires_grad_(True)
        self.dtype, self.device = dtype, device

    def params(self, theta):
        p = torch.cat([self.alpha[:, None], torch.exp(theta[:, :4])], dim=1)
        Es = torch.exp(theta[:, 4])
        y0 = torch.stack([self.M[0].clamp_min(1e-6), torch.zeros_like(Es), self.E[0] / Es, torch.zeros_like(Es)], dim=1)
        return p, y0, Es

    def loss_per_set(self, theta, out=None):
        p, y0, Es = self.params(theta)
        if out is None:
            out = ode.integrate(p.contiguous(), y0.contiguous(), self.dt, self.nsteps, self.every,
                                ckpt_every=100, delta=DELTA)
        m = out[:, :, 0].clamp_min(0.0)
        eps = out[:, :, 2]
        lm = (torch.log1p(m) - torch.log1p(self.M)) ** 2
        le = (eps.abs() * Es - self.E) ** 2 / self.E2
        L = (lm + le).mean(dim=0)
        # a set whose field never screens (|eps| > 1 throughout) grows without
        # bound and overflows: it contributes nothing and is re-seeded
        return torch.where(torch.isfinite(L), L, torch.zeros_like(L))

    def finite(self, theta):
        with torch.no_grad():
            p, y0, Es = self.params(theta)
            out, _ = ode.forward(p.contiguous(), y0.contiguous(), self.dt, self.nsteps, self.every, 0, DELTA)
            L = ((torch.log1p(out[:, :, 0].clamp_min(0.0)) - torch.log1p(self.M)) ** 2).mean(dim=0)
            # runaway sets (multiplicity far beyond any trace) count as overflowed
            return torch.isfinite(L) & (L < 1e4) & torch.isfinite(out).all(dim=2).all(dim=0)

    def reseed(self, ok):
        """Sets that overflowed take the log-parameters of the best finite
        start of their gap, perturbed; a gap with none is drawn afresh."""
        with torch.no_grad():
            L = self.loss_per_set(self.theta)
            L = torch.where(ok, L, torch.full_like(L, float("inf"))).view(self.G, self.starts)
            best = L.argmin(dim=1)
            th = self.theta.view(self.G, self.starts, 5)
            src = th[torch.arange(self.G), best]                       # [G, 5]
            bad = (~ok).view(self.G, self.starts)
            noise = 0.3 * torch.randn_like(th)
            fresh = torch.isinf(L.min(dim=1).values)[:, None, None]
            shift = torch.tensor([1.0, 1.0, 0.0, 0.0, 0.5], dtype=th.dtype, device=th.device)
            new = torch.where(fresh, th + shift, src[:, None, :] + noise)
            th.copy_(torch.where(bad[:, :, None], new, th))
            return int((~ok).sum())

    def loss(self, theta):
        return self.loss_per_set(theta).sum()


def fd_check(prob: Problem, ok, n: int = 8, h: float = 1e-6, seed: int = 1):
    """Largest and median relative difference between the adjoint gradient
    and central differences (step h in the log-parameters) over the five
    log-parameters of n finite sets."""
    g = torch.Generator().manual_seed(seed)
    cand = torch.nonzero(ok.cpu()).flatten()
    idx = cand[torch.randperm(cand.numel(), generator=g)[:n]].to(prob.device)
    th = prob.theta.detach().clone().requires_grad_(True)
    L = prob.loss_per_set(th)
    (grad,) = torch.autograd.grad(L[idx].sum(), th)
    errs = []
    for c in range(5):
        e = torch.zeros_like(th)
        e[:, c] = h
        with torch.no_grad():
            lp = prob.loss_per_set(th + e)[idx]
            lm = prob.loss_per_set(th - e)[idx]
        fd = (lp - lm) / (2 * h)
        ad = grad[idx, c]
        scale = torch.maximum(fd.abs(), ad.abs()).clamp_min(1e-12)
        errs.append((fd - ad).abs() / scale)
    errs = torch.cat(errs)
    return float(errs.max()), float(errs.median())


def run(tr: dict, starts=16, iters=40, lr=0.05, every=50, device="cuda", log=print) -> dict:
    prob = Problem(tr, starts=starts, every=every, device=device)
    opt = torch.optim.Adam([prob.theta], lr=lr)
    hist, times = [], []
    reseeded = 0
    with torch.no_grad():
        med_first = float(prob.loss_per_set(prob.theta.detach()).median())
    for it in range(iters):
        if it % 5 == 0:
            reseeded += prob.reseed(prob.finite(prob.theta))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        opt.zero_grad()
        L = prob.loss(prob.theta)
        L.backward()
        g = prob.theta.grad
        g.copy_(torch.nan_to_num(g, nan=0.0, posinf=0.0, neginf=0.0))
        opt.step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        hist.append(float(L.detach()) / prob.B)
        if log and (it % max(1, iters // 10) == 0 or it == iters - 1):
            log(f"iter {it}: mean loss {hist[-1]:.4g}, {times[-1] * 1e3:.1f} ms (forward + adjoint)")
    ok = prob.finite(prob.theta)
    with torch.no_grad():
        per = prob.loss_per_set(prob.theta)
        per_final = per[ok]
        per = torch.where(ok, per, torch.full_like(per, float("inf"))).view(prob.G, starts)
        best = per.argmin(dim=1)
        th = prob.theta.view(prob.G, starts, 5)[torch.arange(prob.G), best]
    fd, fd_med = fd_check(prob, ok)
    # FP32 forward at the fitted parameters against FP64
    p, y0, Es = prob.params(prob.theta.detach())
    o64, _ = ode.forward(p, y0, prob.dt, prob.nsteps, every, 0, DELTA)
    o32, _ = ode.forward(p.float(), y0.float(), prob.dt.float(), prob.nsteps, every, 0, DELTA)
    m64, m32 = o64[:, ok, 0], o32[:, ok, 0].double()
    rel = ((m32 - m64).abs() / m64.abs().clamp_min(1.0)).max(dim=0).values
    fp32_err = float(rel.max())
    fp32_err_med = float(rel.median())
    fitted = torch.exp(th[:, :4]).cpu().numpy()
    return dict(gaps=prob.G, sets=prob.B, ode_steps=prob.nsteps, iters=iters, reseeded=reseeded,
                finite_sets_final=int(ok.sum()),
                loss_first=hist[0], loss_last=hist[-1], loss_median_first=med_first,
                loss_median_last=float(per_final.median()),
                ms_per_iter_median=float(np.median(times[1:] if len(times) > 1 else times) * 1e3),
                fd_rel_err_max=fd, fd_rel_err_median=fd_med, fp32_vs_fp64_m_rel_err_max=fp32_err,
                fp32_vs_fp64_m_rel_err_median=fp32_err_med,
                best_loss_median=float(per.min(dim=1).values[torch.isfinite(per.min(dim=1).values)].median()),
                fitted_median=dict(t_x=float(np.median(fitted[:, 0])), t_pm=float(np.median(fitted[:, 1])),
                                   t_acc=float(np.median(fitted[:, 2])), g3=float(np.median(fitted[:, 3]))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--traces", required=True)
    ap.add_argument("--starts", type=int, default=16)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    res = run(load_traces(a.traces), starts=a.starts, iters=a.iters, lr=a.lr)
    print(json.dumps(res), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main()
