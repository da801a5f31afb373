"""fit.py on the GPU, for the base model (eq. dis1-dis4) and the extended one
(G = m_pm <gamma^-3> a state): traces made by the model itself at known
parameters are fitted by Adam on the adjoint gradients of the ODE kernels.
The adjoint agrees with central differences, the loss falls from the random
starts, and the fit reports the model's own parameter names."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ES = 3.0
# (parameters of the two gaps, initial state, ODE steps per sample, samples,
# sample interval in t_esc, bounds of the random starts)
CASES = {
    "base": ([[2.0, 5e-3, 4e-3, 5e-8, 5e-7], [3.0, 5e-3, 4e-3, 5e-8, 5e-7]],
             [1.0, 0.0, 1.2, 0.0], 10, 41, 5e-3, None),
    # a point whose stiffness a step of 1e-4 t_esc resolves
    "ext": ([[2.0, 3e-2, 2e-2, 3e-3, 4.0, 30.0], [3.0, 3e-2, 2e-2, 3e-3, 4.0, 30.0]],
            [1.0, 0.0, 1.2, 0.0, 1.0 / 64.0], 10, 81, 1e-3,
            ((1e-2, 1e-1), (1e-2, 1e-1), (1e-3, 1e-2), (2.0, 10.0), (10.0, 100.0))),
}


def _traces(model):
    from paper_2608_21920_b300 import fit, ode
    p, y, every, S, sdt, _ = CASES[model]
    p = torch.tensor(p, dtype=torch.float64, device="cuda")
    y0 = torch.tensor([y, y], dtype=torch.float64, device="cuda")
    dt = torch.full((2,), sdt / every, dtype=torch.float64, device="cuda")
    out, _ = ode.forward(p, y0, dt, (S - 1) * every, every, 0, fit.DELTA, model=model)
    out = out.cpu()
    return dict(M=out[:, :, 0].numpy(), E=(out[:, :, 2].abs() * ES).numpy(), alpha=p[:, 0].cpu().numpy(),
                t_esc=np.ones(2), sample_dt=np.full(2, sdt))


@pytest.mark.parametrize("model", ["base", "ext"])
def test_fit_recovers_a_model_trace(model):
    from paper_2608_21920_b300 import fit
    tr = _traces(model)
    assert tr["M"][-1].min() > 10 * tr["M"][0].max()  # the traces contain a discharge
    _, _, every, _, _, bounds = CASES[model]
    r = fit.run(tr, starts=8, iters=30, lr=0.05, every=every, log=None, model=model, bounds=bounds)
    assert r["model"] == model and r["sets"] == 16
    assert set(r["fitted_median"]) == set(fit.NAMES[model])
    assert r["finite_sets_final"] > 0
    assert r["fd_rel_err_median"] < 1e-5, r
    assert r["loss_median_last"] < r["loss_median_first"], r
    assert all(math.isfinite(v) and v > 0 for v in r["fitted_median"].values())
