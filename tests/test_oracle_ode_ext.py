"""Pins of the oracle's extended concurrency model (the <gamma^-3> moment
equation as a fifth state; Sect. 5.2 names it, App. B/C give its pieces):
each term against a closed form or an independent particle equation."""
import math

import numpy as np
import pytest
import torch

from oracle import ode as OO

BIG = 1e30


def _run(y0, p, dt, n, every=1):
    return OO.rk4_ext(torch.tensor([y0], dtype=torch.float64), torch.tensor([p], dtype=torch.float64), dt, n,
                      record_every=every)[:, 0, :].numpy()


def test_radiation_and_escape_closed_form():
    """No field, no photons: m = m0 e^-t and curvature losses raise every
    particle's gamma^-3 at 3/(gamma_rad^4 t_acc) (eq. dgamma_curv), so
    G(t) = e^-t (G0 + 3 m0 t/(gamma_rad^4 t_acc))."""
    gr, ta, m0, G0 = 10.0, 1e-3, 2.0, 0.05
    out = _run([m0, 0.0, 0.0, 0.0, G0], [0.0, BIG, 1.0, ta, BIG, gr], 1e-3, 2000, every=100)
    t = np.arange(out.shape[0]) * 0.1
    expect = np.exp(-t) * (G0 + 3.0 * m0 * t / (gr ** 4 * ta))
    assert np.allclose(out[:, 4], expect, rtol=1e-11, atol=0)
    assert np.allclose(out[:, 0], m0 * np.exp(-t), rtol=1e-11, atol=0)


def test_pair_birth_closed_form():
    """No field, no new photons, no losses: the photons m_x0 e^-(1 + 1/t_pm)t
    convert into pairs born at gamma_min (eq. gam_inj), so
    m = e^-t (m0 + 2 m_x0 (1 - e^-t/t_pm)) and
    G = e^-t (G0 + 2 m_x0 gamma_min^-3 (1 - e^-t/t_pm))."""
    tpm, gmin, m0, mx0, G0 = 0.3, 2.0, 1.0, 2.0, 0.5
    out = _run([m0, mx0, 0.0, 0.0, G0], [0.0, BIG, tpm, 1e-2, gmin, BIG], 1e-3, 3000, every=100)
    t = np.arange(out.shape[0]) * 0.1
    grow = 1.0 - np.exp(-t / tpm)
    assert np.allclose(out[:, 0], np.exp(-t) * (m0 + 2 * mx0 * grow), rtol=1e-10, atol=0)
    assert np.allclose(out[:, 4], np.exp(-t) * (G0 + 2 * mx0 * gmin ** -3 * grow), rtol=1e-10, atol=0)
    assert np.allclose(out[:, 1], mx0 * np.exp(-(1 + 1 / tpm) * t), rtol=1e-10, atol=0)


def test_cold_beam_matches_a_particle_equation():
    """A single cold stream (no photons): every particle has the same gamma,
    and its energy equation dgamma/dt = eps (j/m)/t_acc - gamma^4/(gamma_rad^4
    t_acc) (the work of the field on the stream, charge times velocity j/m,
    and the curvature losses) gives gamma^-3 = G/m along the model's own
    eps(t), j(t), m(t).  A wrong sign or power in the moment equation fails
    this; the closure is exact for a cold stream."""
    alpha, ta, gr, g0 = 1.5, 1e-2, 8.0, 3.0
    p = torch.tensor([[alpha, BIG, 1.0, ta, BIG, gr]], dtype=torch.float64)
    y = torch.tensor([[1.0, 0.0, 1.0, 0.0, g0 ** -3]], dtype=torch.float64)
    dt, n = 1e-4, 10000

    def f(state):  # the model and the particle's gamma side by side
        yy, g = state[:, :5], state[:, 5]
        m, eps, j = yy[:, 0], yy[:, 2], yy[:, 3]
        dg = eps * (j / m) / ta - g ** 4 / (gr ** 4 * ta)
        return torch.cat([OO.rhs_ext(yy, p), dg[:, None]], dim=1)

    s = torch.cat([y, torch.tensor([[g0]], dtype=torch.float64)], dim=1)
    worst, gmin_seen, gmax_seen = 0.0, g0, g0
    for k in range(n):
        k1 = f(s)
        k2 = f(s + 0.5 * dt * k1)
        k3 = f(s + 0.5 * dt * k2)
        k4 = f(s + dt * k3)
        s = s + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if k % 100 == 99:
            G, m, g = s[0, 4].item(), s[0, 0].item(), s[0, 5].item()
            worst = max(worst, abs(G / m * g ** 3 - 1.0))
            gmin_seen, gmax_seen = min(gmin_seen, g), max(gmax_seen, g)
    assert worst < 1e-9
    assert gmax_seen > 2 * g0  # the stream was accelerated well beyond its start


def test_reduces_to_dis4_while_g3_is_steady():
    """No field work and no losses: pairs born at gamma_min keep G/m at
    gamma_min^-3 when it starts there, and the extended model's (m, m_x,
    eps, j) equal the four-equation model's with g3 = gamma_min^-3 (with
    eps = 0 and alpha = 0 both currents stay zero)."""
    gmin, tpm = 5.0, 0.2
    out = _run([1.0, 1.0, 0.0, 0.0, gmin ** -3], [0.0, BIG, tpm, 1e-3, gmin, BIG], 1e-3, 2000, every=100)
    assert np.allclose(out[:, 4] / out[:, 0], gmin ** -3, rtol=1e-10, atol=0)
    base = OO.rk4(torch.tensor([[1.0, 1.0, 0.0, 0.0]], dtype=torch.float64),
                  torch.tensor([[0.0, BIG, tpm, 1e-3, gmin ** -3]], dtype=torch.float64), 1e-3, 2000,
                  record_every=100)[:, 0, :].numpy()
    assert np.allclose(out[:, :4], base, rtol=1e-13, atol=1e-300)
