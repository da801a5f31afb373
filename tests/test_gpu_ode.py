"""Batched concurrency-model integrator and its hand-written adjoint against
the FP64 oracle (torch CPU RK4), torch autograd and finite differences."""
import numpy as np
import pytest
import torch

from oracle import ode as OO

pytestmark = pytest.mark.gpu


def _sets(B, seed=0, dtype=torch.float64):
    g = torch.Generator().manual_seed(seed)
    u = torch.rand(B, 5, generator=g, dtype=torch.float64)
    p = torch.empty(B, 5, dtype=torch.float64)
    p[:, 0] = 0.5 + 2.0 * u[:, 0]                          # alpha
    p[:, 1] = 10 ** (-3.0 + 1.0 * u[:, 1])                 # t_x
    p[:, 2] = 10 ** (-3.0 + 1.0 * u[:, 2])                 # t_pm
    p[:, 3] = 10 ** (-7.7 + 0.6 * u[:, 3])                 # t_acc
    p[:, 4] = 10 ** (-7.4 + 0.6 * u[:, 4])                 # g3
    y0 = torch.tensor([1.0, 0.0, 1.0, 0.0], dtype=torch.float64).repeat(B, 1)
    dt = torch.full((B,), 2e-4, dtype=torch.float64)
    return p.to(dtype), y0.to(dtype), dt.to(dtype)


def test_forward_matches_oracle_smoothed_gate():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _sets(16)
    out, _ = ode.forward(p.cuda(), y0.cuda(), dt.cuda(), 3000, every=100, delta=1e-2)
    ref = OO.rk4(y0, p, 2e-4, 3000, delta=1e-2, record_every=100)
    rel = ((out.cpu() - ref).abs() / ref.abs().clamp_min(1.0)).max().item()
    assert rel < 1e-10


def test_forward_matches_oracle_hard_gate_first_ignition():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _sets(16, seed=1)
    out, _ = ode.forward(p.cuda(), y0.cuda(), dt.cuda(), 20, every=1, delta=0.0)
    ref = OO.rk4(y0, p, 2e-4, 20, delta=None, record_every=1)
    rel = ((out.cpu() - ref).abs() / ref.abs().clamp_min(1.0)).max().item()
    assert rel < 1e-12


def test_fig2_cycle_on_gpu():
    """The Fig. 2 limit cycle (Sect. 5.5): period 9.1 t_esc within 5%."""
    from paper_2608_21920_b300 import ode
    q = OO.fig2_params()
    p = torch.tensor([[q["alpha"], q["t_x"], q["t_pm"], q["t_acc"], q["g3"]]], dtype=torch.float64)
    y0 = torch.tensor([[1.0, 0.0, 1.0, 0.0]], dtype=torch.float64)
    dt = torch.tensor([2e-4], dtype=torch.float64)
    out, _ = ode.forward(p.cuda(), y0.cuda(), dt.cuda(), 175000, every=5)
    m = out[:, 0, 0].cpu().numpy()
    t = np.arange(m.size) * 1e-3
    i = OO.peaks(t, m)
    i = i[m[i] > 100]
    P = np.diff(t[i][1:]).mean()
    assert abs(P - 9.1) / 9.1 < 0.05
    assert np.all(np.abs(m[i][1:] - 5e3) / 5e3 < 0.5)


def test_adjoint_matches_torch_autograd_fp64():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _sets(8, seed=2)
    n, every = 600, 20
    w = torch.randn(n // every + 1, 8, 4, dtype=torch.float64, generator=torch.Generator().manual_seed(5))
    pc, yc = p.clone().requires_grad_(True), y0.clone().requires_grad_(True)
    ref = OO.rk4(yc, pc, 2e-4, n, delta=1e-2, record_every=every)
    (ref * w).sum().backward()
    pg, yg = p.cuda().requires_grad_(True), y0.cuda().requires_grad_(True)
    out = ode.integrate(pg, yg, dt.cuda(), n, every=every, ckpt_every=37, delta=1e-2)
    (out * w.cuda()).sum().backward()
    for a, b in ((pg.grad.cpu(), pc.grad), (yg.grad.cpu(), yc.grad)):
        rel = ((a - b).abs() / b.abs().clamp_min(1e-30)).max().item()
        assert rel < 1e-9


def test_adjoint_matches_central_differences():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _sets(4, seed=3)
    n, every = 400, 10
    w = torch.randn(n // every + 1, 4, 4, dtype=torch.float64, generator=torch.Generator().manual_seed(9)).cuda()
    pg = p.cuda().requires_grad_(True)
    out = ode.integrate(pg, y0.cuda(), dt.cuda(), n, every=every, ckpt_every=20, delta=1e-2)
    (out * w).sum().backward()
    g = pg.grad.cpu()
    h = 1e-6
    for b in range(4):
        for k in range(5):
            pp, pm = p.clone(), p.clone()
            pp[b, k] *= 1 + h
            pm[b, k] *= 1 - h
            fp = (ode.forward(pp.cuda(), y0.cuda(), dt.cuda(), n, every, 0, 1e-2)[0] * w).sum().item()
            fm = (ode.forward(pm.cuda(), y0.cuda(), dt.cuda(), n, every, 0, 1e-2)[0] * w).sum().item()
            fd = (fp - fm) / (2 * h * p[b, k].item())
            assert abs(fd - g[b, k].item()) <= 1e-6 * max(abs(fd), 1e-3 * g[b].abs().max().item())


def test_fp32_forward_error_bound():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _sets(64, seed=4)
    o64, _ = ode.forward(p.cuda(), y0.cuda(), dt.cuda(), 2000, every=100, delta=1e-2)
    o32, _ = ode.forward(p.float().cuda(), y0.float().cuda(), dt.float().cuda(), 2000, every=100, delta=1e-2)
    rel = ((o32.double() - o64).abs() / o64.abs().clamp_min(1.0)).max().item()
    # FP32 rounding (6e-8 per operation) is amplified by the exponential
    # ignition phase (growth exp(t/t_pm) over 0.4 t_esc with t_pm >= 1e-3)
    # and by the gate switch that follows it; measured 3.5e-2 on B300
    assert rel < 0.1


# ---------------------------------------------------------------- extended model
def _ext_sets(B, seed=0):
    """Parameter sets of the extended model (G = m <gamma^-3> a state) in a
    range whose stiffness 3 eps (j/m) (G/m)^(1/3) / t_acc the step resolves:
    t_acc in [1e-3, 1e-2], gamma_min in [2, 10], gamma_rad in [10, 100]."""
    g = torch.Generator().manual_seed(seed)
    u = torch.rand(B, 6, generator=g, dtype=torch.float64)
    p = torch.empty(B, 6, dtype=torch.float64)
    p[:, 0] = 0.5 + 2.0 * u[:, 0]
    p[:, 1] = 10 ** (-2.0 + 1.0 * u[:, 1])
    p[:, 2] = 10 ** (-2.0 + 1.0 * u[:, 2])
    p[:, 3] = 10 ** (-3.0 + 1.0 * u[:, 3])
    p[:, 4] = 2.0 + 8.0 * u[:, 4]
    p[:, 5] = 10 ** (1.0 + 1.0 * u[:, 5])
    y0 = torch.zeros(B, 5, dtype=torch.float64)
    y0[:, 0], y0[:, 2], y0[:, 4] = 1.0, 1.0, p[:, 4] ** -3
    dt = torch.full((B,), 1e-4, dtype=torch.float64)
    return p, y0, dt


def test_ext_forward_matches_oracle():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _ext_sets(16)
    out, _ = ode.forward(p.cuda(), y0.cuda(), dt.cuda(), 3000, every=100, delta=1e-2, model="ext")
    ref = OO.rk4_ext(y0, p, 1e-4, 3000, delta=1e-2, record_every=100)
    assert torch.isfinite(ref).all()
    rel = ((out.cpu() - ref).abs() / ref.abs().clamp_min(1e-3)).max().item()
    assert rel < 1e-10
    # the inertia measure moved: fresh pairs, acceleration and losses act
    g3 = (ref[:, :, 4] / ref[:, :, 0])
    assert (g3.max(0).values / g3.min(0).values).max().item() > 2.0


def test_ext_adjoint_matches_torch_autograd_fp64():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _ext_sets(8, seed=2)
    n, every = 600, 20
    w = torch.randn(n // every + 1, 8, 5, dtype=torch.float64, generator=torch.Generator().manual_seed(5))
    pc, yc = p.clone().requires_grad_(True), y0.clone().requires_grad_(True)
    ref = OO.rk4_ext(yc, pc, 1e-4, n, delta=1e-2, record_every=every)
    (ref * w).sum().backward()
    pg, yg = p.cuda().requires_grad_(True), y0.cuda().requires_grad_(True)
    out = ode.integrate(pg, yg, dt.cuda(), n, every=every, ckpt_every=37, delta=1e-2, model="ext")
    (out * w.cuda()).sum().backward()
    for a, b in ((pg.grad.cpu(), pc.grad), (yg.grad.cpu(), yc.grad)):
        rel = ((a - b).abs() / b.abs().clamp_min(1e-12 * b.abs().max())).max().item()
        assert rel < 1e-8, rel


def test_ext_adjoint_matches_central_differences():
    from paper_2608_21920_b300 import ode
    p, y0, dt = _ext_sets(4, seed=3)
    n, every = 400, 10
    w = torch.randn(n // every + 1, 4, 5, dtype=torch.float64, generator=torch.Generator().manual_seed(9)).cuda()
    pg = p.cuda().requires_grad_(True)
    out = ode.integrate(pg, y0.cuda(), dt.cuda(), n, every=every, ckpt_every=20, delta=1e-2, model="ext")
    (out * w).sum().backward()
    g = pg.grad.cpu()
    h = 1e-6
    for b in range(4):
        for k in range(6):
            pp, pm = p.clone(), p.clone()
            pp[b, k] *= 1 + h
            pm[b, k] *= 1 - h
            fp = (ode.forward(pp.cuda(), y0.cuda(), dt.cuda(), n, every, 0, 1e-2, model="ext")[0] * w).sum().item()
            fm = (ode.forward(pm.cuda(), y0.cuda(), dt.cuda(), n, every, 0, 1e-2, model="ext")[0] * w).sum().item()
            fd = (fp - fm) / (2 * h * p[b, k].item())
            assert abs(fd - g[b, k].item()) <= 1e-6 * max(abs(fd), 1e-3 * g[b].abs().max().item()), (b, k, fd, g[b, k])
