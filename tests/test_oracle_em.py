"""Pins of the oracle's transverse-field solver (App. A in the 1D reduction):
the Yee scheme against its closed-form discrete modes, the conductor at the
star, the co-rotating frame's virtual current against the static balance it
implies, rotation invariance about h, Gauss's law with the virtual charge,
and the absorbing layer's reflection against Berenger's continuum value.

Equations (code units, c = 1, 4 pi absorbed; d = d/dh):
  dB_y/dt = d E_z, dB_z/dt = -d E_y, dE_y/dt = -d B_z + jv_y,
  dE_z/dt = d B_y + jv_z, and jv_h joins the Ampere step of E_h, with
  jv = -{curl(beta x E) + beta x curl E - curl[beta x (beta x B)]}.
"""
import math

import numpy as np
import pytest

import oracle as O

DX, DT = 0.1, 0.045


def _vacuum(nx, boundary, **kw):
    return O.Sim(nx=nx, dx=kw.pop("dx", DX), dt=kw.pop("dt", DT), boundary=boundary, em=1, **kw)


def test_yee_mode_follows_the_discrete_dispersion():
    """A travelling mode of the leapfrog scheme on the staggered grid:
    sin(omega dt / 2) / dt = sin(k dx / 2) / dx (the textbook Yee relation,
    exact for the discrete equations), E_y = B_z for a wave going up and
    E_z = -B_y for the other polarisation."""
    nx, A = 64, 1e-3
    k = 2 * math.pi * 3 / (nx * DX)
    w = 2 / DT * math.asin(DT / DX * math.sin(k * DX / 2))
    s = _vacuum(nx, O.BC_PERIODIC)
    xc, xi = (np.arange(nx) + 0.5) * DX, np.arange(nx) * DX
    s.set_em(A * np.sin(k * xc + w * DT / 2), -A * np.sin(k * xc + w * DT / 2), A * np.sin(k * xi), A * np.sin(k * xi))
    N = 200
    s.step(N)
    Ey, Ez, By, Bz = s.em()
    ph_e, ph_b = k * xc - w * (N - 0.5) * DT, k * xi - w * N * DT
    assert np.abs(Ey - A * np.sin(ph_e)).max() < 1e-12 * A
    assert np.abs(Ez + A * np.sin(ph_e)).max() < 1e-12 * A
    assert np.abs(Bz - A * np.sin(ph_b)).max() < 1e-12 * A
    assert np.abs(By - A * np.sin(ph_b)).max() < 1e-12 * A
    assert np.abs(s.E()).max() == 0.0  # beta = 0: no virtual current
    # the continuum relation would have drifted by far more than the tolerance
    assert abs(w - k) * N * DT > 1e-3


def test_unit_courant_number_translates_and_the_star_reflects():
    """At dt = dx the 1D Yee scheme moves a wave one cell per step exactly.
    A pulse going down meets the conductor at h = 0 (tangential E = 0) and
    comes back with E_y reversed and B_z unchanged (the method of images)."""
    nx = 200
    s = _vacuum(nx, O.BC_SURFACE, dx=0.1, dt=0.1)
    u = np.exp(-((np.arange(nx + 1) - 100.0) / 6.0) ** 2)
    s.set_em(-u[:nx], np.zeros(nx), np.zeros(nx + 1), u)  # going down: E_y = -B_z
    s.step(60)
    Ey, _, _, Bz = s.em()
    assert np.abs(Bz[: nx + 1 - 60] - u[60:]).max() < 1e-15
    assert np.abs(Ey[: nx - 60] + u[60:nx]).max() < 1e-15
    s.step(140)  # 200 steps: the reflected pulse is back at node 100, going up
    Ey, _, _, Bz = s.em()
    assert np.abs(Bz - u[::-1]).max() < 1e-14
    assert np.abs(Ey - u[::-1][1:]).max() < 1e-14


@pytest.mark.parametrize("beta", [3e-6, 0.3])
def test_virtual_current_drives_the_static_balance(beta):
    """A static E_h = A0 sin(k h) with no particles: jv_y = -beta d E_h drives
    B_z towards App. A's static balance d B_z = jv_y, B_z = -beta E_h (the
    beta^2 terms cancel between jv_y, jv_h and the drift of E_h), around
    which it oscillates at the Yee frequency; jv_h = -beta d E_y moves E_h so
    that E_h - beta B_z stays fixed (Gauss with the virtual charge).  Solving
    the scheme for this one Fourier mode gives
      b_n = -beta A0 (1 - cos(W n dt)) - (dt K)^2 beta A0 sin(W n dt) / (2 sin(W dt)),
    K = 2 sin(k dx / 2) / dx, sin(W dt / 2) = dt K / 2, and E_h = (A0 + beta b_n) sin(k h)."""
    nx, A0 = 64, 0.01
    k = 2 * math.pi * 2 / (nx * DX)
    K = 2 * math.sin(k * DX / 2) / DX
    W = 2 / DT * math.asin(DT * K / 2)
    xi = np.arange(nx) * DX
    for N in (1, 7, 300):
        s = _vacuum(nx, O.BC_PERIODIC, beta_y=beta)
        s.set_E(A0 * np.sin(k * xi))
        s.step(N)
        Ey, Ez, By, Bz = s.em()
        bn = -beta * A0 * (1 - math.cos(W * N * DT)) - (DT * K) ** 2 * beta * A0 * math.sin(W * N * DT) / (
            2 * math.sin(W * DT))
        assert np.abs(Bz - bn * np.sin(k * xi)).max() < 1e-12 * beta * A0
        assert np.abs(s.E() - (A0 + beta * bn) * np.sin(k * xi)).max() < 1e-13 * A0
        assert np.abs(Ez).max() == 0.0 and np.abs(By).max() == 0.0
    # the time average over many periods is the static balance
    s = _vacuum(nx, O.BC_PERIODIC, beta_y=beta)
    s.set_E(A0 * np.sin(k * xi))
    P = 2 * math.pi / W
    n = int(round(20 * P / DT))
    acc = np.zeros(nx)
    for _ in range(n):
        s.step(1)
        acc += s.em()[3]
    i = nx // 8  # sin(k h) = 1 there (k h = pi / 2)
    assert acc[i] / n == pytest.approx(-beta * A0, rel=0.02)


def _pair_plasma(**kw):
    return O.Sim(nx=64, ppc=16, boundary=O.BC_PERIODIC, init=O.INIT_PAIR_THERMAL, theta=0.2, seed_amp=0.05,
                 seed=5, em=1, **kw)


def test_rotation_about_h_rotates_the_transverse_fields():
    """Nothing singles out a direction across h but beta, so turning beta by
    an angle turns (E_y, E_z) and (B_y, B_z) by the same angle and leaves E_h
    and the particles alone: this pins the cross terms of jv."""
    be, th = 0.3, 0.7
    a = _pair_plasma(beta_y=be)
    b = _pair_plasma(beta_y=be * math.cos(th), beta_z=be * math.sin(th))
    a.step(150)
    b.step(150)
    Ey, Ez, By, Bz = a.em()
    Ey2, Ez2, By2, Bz2 = b.em()
    sc = np.abs(Bz).max()
    assert sc > 1e-3 and np.abs(Ez).max() == 0.0 and np.abs(By).max() == 0.0
    for got, want in ((Ey2, math.cos(th) * Ey), (Ez2, math.sin(th) * Ey), (By2, -math.sin(th) * Bz),
                      (Bz2, math.cos(th) * Bz)):
        assert np.abs(got - want).max() < 1e-12 * sc
    assert np.abs(a.E() - b.E()).max() < 1e-13
    assert np.array_equal(a.leptons()["X"], b.leptons()["X"]) or \
        np.abs(a.leptons()["X"] - b.leptons()["X"]).max() < 1e-12


def test_gauss_law_with_the_virtual_charge():
    """d E_h = eta - eta_co - beta_y d B_z + beta_z d B_y holds to round-off
    while jv_h visibly moves E_h (beta = 0.3), in a filtered QED discharge
    at a surface with an absorbing layer (outside the layer), and through the
    merges of a capped one."""
    a = _pair_plasma(beta_y=0.2, beta_z=0.2)
    c = _pair_plasma()
    a.step(150)
    c.step(150)
    r, emax = a.gauss_residual()
    assert r < 1e-14 * max(1.0, emax)
    assert np.abs(a.E() - c.E()).max() > 0.1 * emax  # the coupling is not negligible here
    cfg = dict(nx=256, ppc=4, boundary=O.BC_SURFACE, alpha=2.0, qed=1, b=0.1, lambda_hat=1e-4, rho_hat=20.0,
               rate_mult=20.0, init=O.INIT_COLD, density=1.0, seed=3, em=1, pml_cells=16, beta_y=3e-3,
               filter_passes=8, inject_theta=0.3)
    s = O.Sim(**cfg)
    s.step(400)
    r, emax = s.gauss_residual()
    assert r < 1e-13 * max(1.0, emax)
    assert np.abs(s.em()[0]).max() > 1e-4
    # through merges under a cap (their re-centring flux reaches E_h), oblique beta
    s = O.Sim(**dict(cfg, filter_passes=0, inject_theta=0.0, beta_y=0.05, beta_z=0.03, cap=450))
    s.step(900)
    r, emax = s.gauss_residual()
    assert s.counters()["merged"] > 0 and r < 1e-13 * max(1.0, emax)


def _pml_run(nx, pml, n):
    s = _vacuum(nx, O.BC_SURFACE, pml_cells=pml)
    xc, xi = (np.arange(nx) + 0.5) * DX, np.arange(nx + 1) * DX
    x0, W = 250 * DX, 8 * DX
    f = lambda x: np.exp(-((x - x0) / W) ** 2)  # noqa: E731
    s.set_em(f(xc + DT / 2), np.zeros(nx), np.zeros(nx + 1), f(xi))  # going up: E_y = B_z
    s.step(n)
    return s.em()


def test_absorbing_layer_reflects_what_its_grading_predicts():
    """A unit pulse runs into the layer at the top and what comes back is
    measured against the same run on a domain long enough that nothing
    returns.  Berenger's matched layer with sigma ~ x^3 reflects
    exp(-2 sigma_max L / 4) = 1e-6 in the continuum (the default sigma_max);
    the discrete layer approaches it as it thickens, against total
    reflection from the bare conductor."""
    n = int((2 * (40 - 25) + 6) / DT)
    ref = _pml_run(1600, 0, n)
    out = {}
    for pml in (0, 8, 16, 32):
        a = _pml_run(400, pml, n)
        m = 400 - pml
        out[pml] = max(np.abs(a[0][:m] - ref[0][:m]).max(), np.abs(a[3][:m] - ref[3][:m]).max())
    assert out[0] > 0.9
    assert out[8] < 1e-4 and out[16] < 1e-5
    assert 0.5e-6 < out[32] < 2e-6


def test_discharge_field_spectrum_and_transverse_level():
    """Three statements of Sect. 6.6 about the discharge (order-of-magnitude
    checks; the run is config 1 of the workloads at the paper's beta = 3e-6):
    the oscillations reach delta E_h / E_rot ~ 1e-2 (E_rot = |eta_co| H_gap
    in code units; delta E_h the field less its 16-cell running mean, largest
    over the run within a decade of 1e-2), the power spectrum of E_h over the
    gap falls as k^-2 (the fitted slope within [-2.7, -1.7] over the resolved
    band), and the rotating frame's E_y stays about a millionth of E_h (the
    median over the run of max |E_y| / max |E_h| within a decade of 1e-6)."""
    from tests import _pair as P
    cfg = dict(P.CONFIG1, em=1, beta_y=3e-6, pml_cells=32)
    s = O.Sim(**{k: v for k, v in cfg.items() if k in O.DEFAULTS})
    Hc = int(0.8 * cfg["nx"])
    E_rot = 0.8 * cfg["nx"] * cfg["dx"]
    ratios, spec, osc = [], [], []
    w = np.hanning(Hc)
    for blk in range(40):
        s.step(100)
        E, Ey = s.E()[:Hc], s.em()[0][:Hc]
        ratios.append(np.abs(Ey).max() / np.abs(E).max())
        osc.append(np.abs((E - np.convolve(E, np.ones(16) / 16, mode="same"))[16:-16]).max() / E_rot)
        if blk >= 20:  # after ignition (pairs from about step 300)
            spec.append(np.abs(np.fft.rfft((E - E.mean()) * w)) ** 2)
    assert s.counters()["pairs"] > 1000
    S = np.mean(spec, axis=0)
    k = np.arange(S.size)
    band = (k >= 8) & (k <= 150)
    slope = np.polyfit(np.log(k[band]), np.log(S[band]), 1)[0]
    assert -2.7 < slope < -1.7, slope
    assert 1e-7 < np.median(ratios) < 1e-5, np.median(ratios)
    assert 1e-3 < max(osc) < 1e-1, max(osc)


def test_the_papers_full_setup_keeps_gauss_law():
    """Every option of Sect. 6.1 at once: the start with protons (the linear
    ramp), QED, the 8-pass current filter, the T = 0.3 atmosphere, the
    co-rotating frame at beta = 3e-6 with an absorbing layer.  Gauss's law
    (smoothed charge with protons, virtual charge) holds to round-off over a
    discharge, and E_y stays of order beta E_h."""
    cfg = dict(nx=256, ppc=4, dx=0.1, dt=0.045, alpha=2.0, b=0.1, qed=1, lambda_hat=2e-4, rho_hat=10.0,
               rate_mult=5.0, init=O.INIT_GAP_PROTONS, boundary=O.BC_SURFACE, seed=3, protons=1, filter_passes=8,
               inject_theta=0.3, em=1, beta_y=3e-6, pml_cells=32)
    s = O.Sim(**cfg)
    r, emax = s.gauss_residual()
    assert r < 1e-13 * max(1.0, emax)
    s.step(1500)
    c = s.counters()
    assert c["pairs"] > 1000 and c["injected"] > 0
    assert (s.leptons()["heavy"] == 1).sum() > 100
    r, emax = s.gauss_residual()
    assert r < 1e-12 * max(1.0, emax)
    ratio = np.abs(s.em()[0]).max() / emax
    assert 1e-7 < ratio < 1e-4, ratio
