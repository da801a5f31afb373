"""fit.py's host logic on the CPU: the fit's integrator (the GPU kernels of
ode.py) is replaced, inside this test only, by the oracle's torch RK4, so
that the parameter mapping, the loss, the gradient path and the re-seeding
of overflowed sets can be checked without a GPU.  Traces are made by the
same model at known parameters."""
import math

import numpy as np
import pytest
import torch

from oracle import ode as oracle_ode

TRUTH = dict(alpha=2.0, t_x=5e-3, t_pm=4e-3, t_acc=5e-8, g3=5e-7)
ES = 3.0          # the field scale of the traces
EVERY, S = 10, 41  # ODE steps per sample, samples
SAMPLE_DT = 5e-3   # in t_esc


@pytest.fixture
def fit(monkeypatch):
    from paper_2608_21920_b300 import fit as F
    from paper_2608_21920_b300 import ode as O

    def forward(p, y0, dt, nsteps, every=1, ckpt_every=0, delta=0.0, model="base"):
        rk = oracle_ode.rk4 if model == "base" else oracle_ode.rk4_ext
        return rk(y0, p, dt[:, None], nsteps, delta=delta or None, record_every=every), None

    def integrate(p, y0, dt, nsteps, every=1, ckpt_every=None, delta=0.0, model="base"):
        return forward(p, y0, dt, nsteps, every, 0, delta, model)[0]

    monkeypatch.setattr(O, "forward", forward)
    monkeypatch.setattr(O, "integrate", integrate)
    return F


def _traces(fit):
    p = oracle_ode.as_tensor([TRUTH, dict(TRUTH, alpha=3.0)])
    y0 = torch.tensor([[1.0, 0.0, 1.2, 0.0]] * 2, dtype=torch.float64)
    dt = torch.full((2,), SAMPLE_DT / EVERY, dtype=torch.float64)
    out = oracle_ode.rk4(y0, p, dt[:, None], (S - 1) * EVERY, delta=fit.DELTA, record_every=EVERY)
    M = out[:, :, 0].numpy()
    E = (out[:, :, 2].abs() * ES).numpy()
    return dict(M=M, E=E, alpha=np.array([2.0, 3.0]), t_esc=np.ones(2), sample_dt=np.full(2, SAMPLE_DT))


def _truth_theta(prob):
    th = torch.tensor([math.log(TRUTH[k]) for k in ("t_x", "t_pm", "t_acc", "g3")] + [math.log(ES)],
                      dtype=torch.float64)
    return th.repeat(prob.B, 1)


def test_loss_vanishes_at_the_generating_parameters(fit):
    tr = _traces(fit)
    assert tr["M"][-1].min() > 10 * tr["M"][0].max()  # the traces contain a discharge
    prob = fit.Problem(tr, starts=3, every=EVERY, device="cpu")
    L = prob.loss_per_set(_truth_theta(prob))
    assert L.max() < 1e-20
    L0 = prob.loss_per_set(prob.theta.detach())
    ok = prob.finite(prob.theta)
    assert ok.any() and L0[ok].min() > 1e-6  # random starts are not already at the answer
    assert torch.all(L0[~ok] == 0.0)  # an overflowing start contributes nothing (it is re-seeded)


def test_gradient_matches_central_differences(fit):
    prob = fit.Problem(_traces(fit), starts=3, every=EVERY, device="cpu")
    with torch.no_grad():
        prob.theta.copy_(_truth_theta(prob) + 0.05 * torch.randn(prob.B, 5, dtype=torch.float64,
                                                                   generator=torch.Generator().manual_seed(3)))
    ok = prob.finite(prob.theta)
    assert bool(ok.all())
    mx, med = fit.fd_check(prob, ok, n=4, h=1e-6)
    assert med < 1e-5 and mx < 1e-3


def test_reseed_replaces_only_the_flagged_sets(fit):
    prob = fit.Problem(_traces(fit), starts=3, every=EVERY, device="cpu")
    before = prob.theta.detach().clone()
    ok = torch.tensor([True, False, True, True, True, False])
    n = prob.reseed(ok)
    after = prob.theta.detach()
    assert n == 2
    assert torch.equal(after[ok], before[ok])
    assert not torch.equal(after[~ok], before[~ok])
    # a flagged set starts from its own gap's best finite start, perturbed
    L = prob.loss_per_set(before).view(2, 3)
    for bad, gap in ((1, 0), (5, 1)):
        cand = [i for i in range(3 * gap, 3 * gap + 3) if ok[i]]
        best = min(cand, key=lambda i: float(L.view(-1)[i]))
        assert float((after[bad] - before[best]).abs().max()) < 2.0


def test_load_traces_takes_t_esc_from_the_gap_length(tmp_path):
    """The model's time unit is H_gap / c (Sect. 5.2): a trace saved with an
    explicit gap length uses it, one saved with 0 falls back to 0.8 nx dx."""
    from paper_2608_21920_b300 import fit
    p = tmp_path / "tr.npz"
    np.savez(p, M_avg=np.ones((3, 2)), E_abs_max=np.ones((3, 2)), step=np.array([0, 10, 20]),
             param_nx=np.array([100.0, 200.0]), param_dx=np.array([0.1, 0.1]), param_dt=np.array([0.045, 0.045]),
             param_alpha=np.array([1.0, 2.0]), param_gap_length=np.array([5.0, 0.0]))
    tr = fit.load_traces(str(p))
    assert np.allclose(tr["t_esc"], [5.0, 16.0])
    assert np.allclose(tr["sample_dt"], 0.45)


# ---------------------------------------------------------------- extended model
# a point of the extended model whose stiffness a step of 1e-4 t_esc resolves
TRUTH_EXT = dict(alpha=2.0, t_x=3e-2, t_pm=2e-2, t_acc=3e-3, gamma_min=4.0, gamma_rad=30.0)
BOUNDS_EXT = ((1e-2, 1e-1), (1e-2, 1e-1), (1e-3, 1e-2), (2.0, 10.0), (10.0, 100.0))
EVERY_EXT, S_EXT, SAMPLE_DT_EXT = 10, 81, 1e-3


def _traces_ext(fit):
    keys = ("alpha", "t_x", "t_pm", "t_acc", "gamma_min", "gamma_rad")
    p = torch.tensor([[TRUTH_EXT[k] for k in keys], [3.0] + [TRUTH_EXT[k] for k in keys[1:]]], dtype=torch.float64)
    m0 = 1.0
    y0 = torch.tensor([[m0, 0.0, 1.2, 0.0, m0 * TRUTH_EXT["gamma_min"] ** -3]] * 2, dtype=torch.float64)
    dt = torch.full((2, 1), SAMPLE_DT_EXT / EVERY_EXT, dtype=torch.float64)
    out = oracle_ode.rk4_ext(y0, p, dt, (S_EXT - 1) * EVERY_EXT, delta=fit.DELTA, record_every=EVERY_EXT)
    return dict(M=out[:, :, 0].numpy(), E=(out[:, :, 2].abs() * ES).numpy(), alpha=np.array([2.0, 3.0]),
                t_esc=np.ones(2), sample_dt=np.full(2, SAMPLE_DT_EXT))


def _truth_theta_ext(prob):
    th = torch.tensor([math.log(TRUTH_EXT[k]) for k in ("t_x", "t_pm", "t_acc", "gamma_min", "gamma_rad")]
                      + [math.log(ES)], dtype=torch.float64)
    return th.repeat(prob.B, 1)


def test_ext_problem_has_the_extended_parameters(fit):
    prob = fit.Problem(_traces_ext(fit), starts=3, every=EVERY_EXT, device="cpu", model="ext", bounds=BOUNDS_EXT)
    assert prob.theta.shape == (6, 6)
    p, y0, Es = prob.params(_truth_theta_ext(prob))
    assert p.shape == (6, 6) and y0.shape == (6, 5)
    assert torch.allclose(p[0, 1:], torch.tensor([3e-2, 2e-2, 3e-3, 4.0, 30.0], dtype=torch.float64))
    # the plasma present at the start carries gamma_min^-3
    assert torch.allclose(y0[:, 4], y0[:, 0] / 64.0)
    assert torch.allclose(Es, torch.full((6,), ES, dtype=torch.float64))
    # draws inside the given bounds
    lo = torch.tensor([math.log(b[0]) for b in BOUNDS_EXT], dtype=torch.float64)
    hi = torch.tensor([math.log(b[1]) for b in BOUNDS_EXT], dtype=torch.float64)
    th = prob.theta.detach()[:, :5]
    assert bool(((th >= lo) & (th <= hi)).all())
    with pytest.raises(ValueError):
        fit.Problem(_traces_ext(fit), starts=1, every=EVERY_EXT, device="cpu", model="other")


def test_ext_loss_vanishes_at_the_generating_parameters(fit):
    tr = _traces_ext(fit)
    assert tr["M"][-1].min() > 10 * tr["M"][0].max()  # the traces contain a discharge
    prob = fit.Problem(tr, starts=3, every=EVERY_EXT, device="cpu", model="ext", bounds=BOUNDS_EXT)
    assert prob.loss_per_set(_truth_theta_ext(prob)).max() < 1e-20
    # the base model fitted to the same traces cannot reproduce them exactly
    base = fit.Problem(tr, starts=3, every=EVERY_EXT, device="cpu")
    th = torch.tensor([math.log(v) for v in (3e-2, 2e-2, 3e-3, 4.0 ** -3, ES)], dtype=torch.float64).repeat(6, 1)
    assert base.loss_per_set(th).min() > 1e-8


def test_ext_gradient_matches_central_differences(fit):
    prob = fit.Problem(_traces_ext(fit), starts=2, every=EVERY_EXT, device="cpu", model="ext", bounds=BOUNDS_EXT)
    with torch.no_grad():
        prob.theta.copy_(_truth_theta_ext(prob) + 0.05 * torch.randn(prob.B, 6, dtype=torch.float64,
                                                                       generator=torch.Generator().manual_seed(4)))
    ok = prob.finite(prob.theta)
    assert bool(ok.all())
    mx, med = fit.fd_check(prob, ok, n=2, h=1e-6)
    assert med < 1e-5 and mx < 1e-3


def test_ext_reseed_keeps_the_width(fit):
    prob = fit.Problem(_traces_ext(fit), starts=3, every=EVERY_EXT, device="cpu", model="ext", bounds=BOUNDS_EXT)
    before = prob.theta.detach().clone()
    ok = torch.tensor([True, True, False, True, True, True])
    assert prob.reseed(ok) == 1
    after = prob.theta.detach()
    assert after.shape == before.shape
    assert torch.equal(after[ok], before[ok]) and not torch.equal(after[2], before[2])
