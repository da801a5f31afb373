"""FP64 reference integrator of the discharge concurrency model.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The model is the four-ODE system of Sect. 5.2 (eq. dis1 to dis4), in units of
t_esc = 1:

    dm_pm/dt = 2 m_x / t_pm - m_pm
    dm_x/dt  = -m_x / t_pm + H(|eps| - 1) m_pm / t_x - m_x
    deps/dt  = alpha - j
    dj/dt    = -j + m_pm eps g3 / t_acc

State y = (m_pm, m_x, eps, j); parameters p = (alpha, t_x, t_pm, t_acc, g3).
H is the Heaviside gate; for differentiation the smoothed gate
H_delta(z) = (1 + tanh(z/delta))/2 replaces it (a reading: the hard gate has
no derivative at its switching times).

Classical fourth-order Runge-Kutta with a fixed step, in plain torch FP64 on
the CPU, so that torch autograd gives the reference gradient.
"""
from __future__ import annotations

import numpy as np
import torch


def gate(z, delta):
    if delta is None or delta == 0.0:
        return (z > 0).to(z.dtype)
    return 0.5 * (1.0 + torch.tanh(z / delta))


def rhs(y, p, delta=None):
    """Right-hand side of eq. dis1-dis4 for a batch: y [B,4], p [B,5]."""
    m, mx, eps, j = y[:, 0], y[:, 1], y[:, 2], y[:, 3]
    alpha, tx, tpm, tacc, g3 = p[:, 0], p[:, 1], p[:, 2], p[:, 3], p[:, 4]
    H = gate(torch.abs(eps) - 1.0, delta)
    dm = 2.0 * mx / tpm - m
    dmx = -mx / tpm + H * m / tx - mx
    deps = alpha - j
    dj = -j + m * eps * g3 / tacc
    return torch.stack([dm, dmx, deps, dj], dim=1)


def rk4(y0, p, dt, nsteps, delta=None, record_every=1):
    """Integrate from y0 for nsteps steps of size dt; returns the states at
    steps 0, record_every, 2*record_every, ... as a tensor [T, B, 4]."""
    y = y0
    out = [y]
    for n in range(nsteps):
        k1 = rhs(y, p, delta)
        k2 = rhs(y + 0.5 * dt * k1, p, delta)
        k3 = rhs(y + 0.5 * dt * k2, p, delta)
        k4 = rhs(y + dt * k3, p, delta)
        y = y + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if (n + 1) % record_every == 0:
            out.append(y)
    return torch.stack(out, dim=0)


# --------------------------------------------------------------------------
# Extended model: the plasma-inertia measure as a state.  Sect. 5.2 says the
# paper solved a model with <gamma^-3> obtained by a moment expansion of the
# 1D Vlasov equation but does not give it; this is one such moment, in the
# paper's own approximations, with each closure stated:
#
#  * the moment of <gamma^-3> over the pair plasma, G = m_pm <gamma^-3>,
#    escapes like m_pm (c d/dh -> c/L, the rate 1/t_esc = 1);
#  * acceleration by the field: du/dt = eps/t_acc per unit charge along the
#    force (the t_acc of eq. dis4), so d<gamma^-3>/dt = -3 <gamma^-4 q beta>
#    eps/t_acc; the cold-beam closure <gamma^-4 q beta> = <gamma^-3>^(4/3)
#    j/m_pm (one Lorentz factor per stream, beta -> 1 with the sign of the
#    current) gives dG/dt = -3 eps j (G/m_pm)^(4/3) / t_acc;
#  * curvature losses (eq. dgamma_curv): dgamma/dt = -gamma^4/(gamma_rad^4
#    t_acc), gamma_rad where they balance the acceleration at eps = 1
#    (eq. gam_rad), so d<gamma^-3>/dt = +3/(gamma_rad^4 t_acc) per particle;
#  * pairs are born at gamma_min (eq. gam_inj) at the rate 2 m_x/t_pm of
#    eq. dis1, bringing 2 gamma_min^-3 m_x/t_pm to G;
#  * eq. dis4 with m_pm <gamma^-3> = G: dj/dt = -j + eps G/t_acc.
#
# State y = (m_pm, m_x, eps, j, G); parameters p = (alpha, t_x, t_pm, t_acc,
# gamma_min, gamma_rad).  (G/m)^(4/3) is taken of max(G, 0).

def rhs_ext(y, p, delta=None):
    """Right-hand side of the extended model for a batch: y [B,5], p [B,6]."""
    m, mx, eps, j, G = y[:, 0], y[:, 1], y[:, 2], y[:, 3], y[:, 4]
    alpha, tx, tpm, tacc, gmin, grad = (p[:, i] for i in range(6))
    H = gate(torch.abs(eps) - 1.0, delta)
    g3 = torch.clamp(G, min=0.0) / m
    dm = 2.0 * mx / tpm - m
    dmx = -mx / tpm + H * m / tx - mx
    deps = alpha - j
    dj = -j + eps * G / tacc
    dG = (2.0 * mx / tpm) * gmin ** -3 - G - 3.0 * eps * j * g3 ** (4.0 / 3.0) / tacc + 3.0 * m / (grad ** 4 * tacc)
    return torch.stack([dm, dmx, deps, dj, dG], dim=1)


def rk4_ext(y0, p, dt, nsteps, delta=None, record_every=1):
    """RK4 of the extended model; states at steps 0, record_every, ... [T, B, 5]."""
    y = y0
    out = [y]
    for n in range(nsteps):
        k1 = rhs_ext(y, p, delta)
        k2 = rhs_ext(y + 0.5 * dt * k1, p, delta)
        k3 = rhs_ext(y + 0.5 * dt * k2, p, delta)
        k4 = rhs_ext(y + dt * k3, p, delta)
        y = y + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if (n + 1) % record_every == 0:
            out.append(y)
    return torch.stack(out, dim=0)


def fig2_params():
    """Fig. 2 (Sect. 5.5): alpha = 2, t_x = t_pm = 1e-3, t_acc = 4e-8, g3 = 8e-8."""
    return dict(alpha=2.0, t_x=1e-3, t_pm=1e-3, t_acc=4e-8, g3=8e-8)


def as_tensor(params_list, dtype=torch.float64):
    return torch.tensor([[q["alpha"], q["t_x"], q["t_pm"], q["t_acc"], q["g3"]]
                         for q in params_list], dtype=dtype)


def peaks(t, m):
    """Local maxima of a sampled trace: indices i with m[i-1] < m[i] >= m[i+1]."""
    m = np.asarray(m)
    i = np.where((m[1:-1] > m[:-2]) & (m[1:-1] >= m[2:]))[0] + 1
    return i


def rk4_scalar(y0, q, dt, nsteps, record_every=1):
    """Single parameter set in plain Python floats (fast for long pins).
    q = dict(alpha, t_x, t_pm, t_acc, g3); hard Heaviside gate.
    Returns (t, Y) with Y of shape [T, 4]."""
    a, tx, tpm, tacc, g3 = q["alpha"], q["t_x"], q["t_pm"], q["t_acc"], q["g3"]

    def f(m, mx, e, j):
        H = 1.0 if abs(e) - 1.0 > 0.0 else 0.0
        return (2.0 * mx / tpm - m, -mx / tpm + H * m / tx - mx, a - j, -j + m * e * g3 / tacc)

    m, mx, e, j = (float(v) for v in y0)
    ts, out = [0.0], [(m, mx, e, j)]
    h2, h6 = 0.5 * dt, dt / 6.0
    for n in range(nsteps):
        k1 = f(m, mx, e, j)
        k2 = f(m + h2 * k1[0], mx + h2 * k1[1], e + h2 * k1[2], j + h2 * k1[3])
        k3 = f(m + h2 * k2[0], mx + h2 * k2[1], e + h2 * k2[2], j + h2 * k2[3])
        k4 = f(m + dt * k3[0], mx + dt * k3[1], e + dt * k3[2], j + dt * k3[3])
        m += h6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        mx += h6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        e += h6 * (k1[2] + 2 * k2[2] + 2 * k3[2] + k4[2])
        j += h6 * (k1[3] + 2 * k2[3] + 2 * k3[3] + k4[3])
        if (n + 1) % record_every == 0:
            ts.append((n + 1) * dt)
            out.append((m, mx, e, j))
    return np.array(ts), np.array(out)
