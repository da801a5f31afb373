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

With model="ext" the fitted model is the extended one, G = m_pm <gamma^-3>
a fifth state (ode.py): ln gamma_min (the pair-birth Lorentz factor, eq.
gam_inj) and ln gamma_rad (the radiation-limited one, eq. gam_rad) replace
ln g3, drawn over gamma_min in [1e2, 1e3] and gamma_rad in [1e6, 1e8], and the
plasma present at the start carries gamma_min^-3 too: G(0) = m(0)
gamma_min^-3.  The extended model is stiff near the Fig. 2 point (steps of a
few 1e-6 t_esc), so `every` (ODE steps per trace sample) has to be large.

    python -m paper_2608_21920_b300.fit --traces batch.npz --starts 16 --iters 40
    python -m paper_2608_21920_b300.fit --traces batch.npz --model ext --every 2000
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
# t_x, t_pm, t_acc, gamma_min, gamma_rad
BOUNDS_EXT = ((1e-4, 1e-2), (1e-4, 1e-2), (1e-8, 1e-7), (1e2, 1e3), (1e6, 1e8))
NAMES = {"base": ("t_x", "t_pm", "t_acc", "g3"), "ext": ("t_x", "t_pm", "t_acc", "gamma_min", "gamma_rad")}


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
    """The batched fit: B = gaps x starts parameter sets; theta [B, K + 1]
    holds the K log-parameters of the model (NAMES[model]) and ln E_s."""

    def __init__(self, tr: dict, starts: int = 16, every: int = 50, seed: int = 0,
                 dtype=torch.float64, device="cuda", model: str = "base", bounds=None):
        if model not in NAMES:
            raise ValueError(f"model {model!r}: 'base' or 'ext'")
        bounds = bounds or (BOUNDS if model == "base" else BOUNDS_EXT)
        assert len(bounds) == len(NAMES[model])
        self.model, self.K = model, len(bounds)
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
        lo = torch.tensor([math.log(b[0]) for b in bounds], dtype=dtype)
        hi = torch.tensor([math.log(b[1]) for b in bounds], dtype=dtype)
        th = lo + (hi - lo) * torch.rand(self.B, self.K, generator=g, dtype=dtype)
        Emax = self.E.max(dim=0).values.cpu().clamp_min(1e-12)
        lnEs = torch.log(Emax / 2.0) + 0.5 * torch.randn(self.B, generator=g, dtype=dtype)
        self.theta = torch.cat([th, lnEs[:, None]], dim=1).to(device).requires_grad_(True)
        self.dtype, self.device = dtype, device

    def params(self, theta):
        K = self.K
        p = torch.cat([self.alpha[:, None], torch.exp(theta[:, :K])], dim=1)
        Es = torch.exp(theta[:, K])
        m0 = self.M[0].clamp_min(1e-6)
        y = [m0, torch.zeros_like(Es), self.E[0] / Es, torch.zeros_like(Es)]
        if self.model == "ext":
            y.append(m0 * torch.exp(-3.0 * theta[:, 3]))  # G(0) = m(0) gamma_min^-3
        return p, torch.stack(y, dim=1), Es

    def loss_per_set(self, theta, out=None):
        p, y0, Es = self.params(theta)
        if out is None:
            out = ode.integrate(p.contiguous(), y0.contiguous(), self.dt, self.nsteps, self.every,
                                ckpt_every=100, delta=DELTA, model=self.model)
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
            out, _ = ode.forward(p.contiguous(), y0.contiguous(), self.dt, self.nsteps, self.every, 0, DELTA,
                                 model=self.model)
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
            th = self.theta.view(self.G, self.starts, self.K + 1)
            src = th[torch.arange(self.G), best]                       # [G, K + 1]
            bad = (~ok).view(self.G, self.starts)
            noise = 0.3 * torch.randn_like(th)
            fresh = torch.isinf(L.min(dim=1).values)[:, None, None]
            # a gap with no finite start: slower pair production, smaller field scale
            shift = torch.zeros(self.K + 1, dtype=th.dtype, device=th.device)
            shift[0], shift[1], shift[self.K] = 1.0, 1.0, 0.5
            new = torch.where(fresh, th + shift, src[:, None, :] + noise)
            th.copy_(torch.where(bad[:, :, None], new, th))
            return int((~ok).sum())

    def loss(self, theta):
        return self.loss_per_set(theta).sum()


def fd_check(prob: Problem, ok, n: int = 8, h: float = 1e-6, seed: int = 1):
    """Largest and median relative difference between the adjoint gradient
    and central differences (step h in the log-parameters) over all the
    log-parameters (the model's and ln E_s) of n finite sets."""
    g = torch.Generator().manual_seed(seed)
    cand = torch.nonzero(ok.cpu()).flatten()
    idx = cand[torch.randperm(cand.numel(), generator=g)[:n]].to(prob.device)
    th = prob.theta.detach().clone().requires_grad_(True)
    L = prob.loss_per_set(th)
    (grad,) = torch.autograd.grad(L[idx].sum(), th)
    errs = []
    for c in range(prob.K + 1):
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


def run(tr: dict, starts=16, iters=40, lr=0.05, every=50, device="cuda", log=print, model="base",
        bounds=None) -> dict:
    prob = Problem(tr, starts=starts, every=every, device=device, model=model, bounds=bounds)
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
        th = prob.theta.view(prob.G, starts, prob.K + 1)[torch.arange(prob.G), best]
    fd, fd_med = fd_check(prob, ok)
    # FP32 forward at the fitted parameters against FP64
    p, y0, Es = prob.params(prob.theta.detach())
    o64, _ = ode.forward(p, y0, prob.dt, prob.nsteps, every, 0, DELTA, model=model)
    o32, _ = ode.forward(p.float(), y0.float(), prob.dt.float(), prob.nsteps, every, 0, DELTA, model=model)
    m64, m32 = o64[:, ok, 0], o32[:, ok, 0].double()
    rel = ((m32 - m64).abs() / m64.abs().clamp_min(1.0)).max(dim=0).values
    fp32_err = float(rel.max())
    fp32_err_med = float(rel.median())
    fitted = torch.exp(th[:, :prob.K]).cpu().numpy()
    return dict(model=model, gaps=prob.G, sets=prob.B, ode_steps=prob.nsteps, iters=iters, reseeded=reseeded,
                finite_sets_final=int(ok.sum()),
                loss_first=hist[0], loss_last=hist[-1], loss_median_first=med_first,
                loss_median_last=float(per_final.median()),
                ms_per_iter_median=float(np.median(times[1:] if len(times) > 1 else times) * 1e3),
                fd_rel_err_max=fd, fd_rel_err_median=fd_med, fp32_vs_fp64_m_rel_err_max=fp32_err,
                fp32_vs_fp64_m_rel_err_median=fp32_err_med,
                best_loss_median=float(per.min(dim=1).values[torch.isfinite(per.min(dim=1).values)].median()),
                fitted_median={k: float(np.median(fitted[:, i])) for i, k in enumerate(NAMES[model])})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--traces", required=True)
    ap.add_argument("--starts", type=int, default=16)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--every", type=int, default=50, help="ODE steps per trace sample")
    ap.add_argument("--model", default="base", choices=sorted(NAMES))
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    res = run(load_traces(a.traces), starts=a.starts, iters=a.iters, lr=a.lr, every=a.every, model=a.model)
    print(json.dumps(res), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main()
