"""Pins of the oracle's transverse particle current (App. A; Sect. 6.6,
Fig. 8) in the guiding-centre limit of the strong field: with B = B_* h-hat
+ B_perp and B_* = b / lambda_hat (omega_B / omega_p in code units), a
particle slides along its field line at beta_h and drifts at E x B / B^2:

    v_y = (beta_h B_y + E_z) / B_*,   v_z = (beta_h B_z - E_y) / B_*,

deposited from the start-of-step position with the unit top-hat cloud on
cells, j_perp(c) = sum q w v_perp S_c / dx, and entering the cells' update
as dE_perp/dt = ... - j_perp.  The values below are worked by hand from
those definitions: one particle, a frame at rest (no virtual current) and
uniform fields, so that each step's change of E_perp is -dt j_perp alone.
A plausible slip (the drift's sign, E_y and E_z swapped, a missing 1/B_*,
1/dx or charge, the cloud put on the wrong cells, a mass in the drift)
fails one of them.
"""
import math

import numpy as np
import pytest

import oracle as O

DX, DT = 0.5, 0.05
B_, LAM = 0.2, 0.02        # B_* = b / lambda_hat = 10
BS = B_ / LAM


def _sim(nx=16, boundary=O.BC_PERIODIC, **kw):
    s = O.Sim(nx=nx, dx=DX, dt=DT, boundary=boundary, em=1, jperp=1, b=B_, lambda_hat=LAM, **kw)
    s.set_E(np.zeros(s.nnode))
    return s


def _uniform(s, Ey=0.0, Ez=0.0, By=0.0, Bz=0.0):
    nx, nn = s.cfg["nx"], s.nnode
    s.set_em(np.full(nx, Ey), np.full(nx, Ez), np.full(nn, By), np.full(nn, Bz))


def test_drift_of_an_electron_at_rest_in_a_uniform_E_y():
    """u = 0 and E_h = 0: the electron stays at rest and drifts at
    v_z = -E_y / B_* = -0.03; its cloud, centred on cell 4, is all in cell
    4: j_z = q w v_z / dx = (-1)(0.2)(-0.03)/0.5 = 0.012, so E_z[4] =
    -dt 0.012, and B_y at the nodes of cell 4 follows it in the same step."""
    s = _sim()
    _uniform(s, Ey=0.3)
    s.add_lepton(1, -1, 4.5, 0.0, 0.2)
    s.step(1)
    Jy, Jz = s.jperp()
    assert Jz[4] == pytest.approx(0.012, rel=1e-14)
    assert np.count_nonzero(Jz) == 1 and np.count_nonzero(Jy) == 0
    Ey, Ez, By, Bz = s.em()
    assert Ez[4] == pytest.approx(-DT * 0.012, rel=1e-14)
    assert np.count_nonzero(Ez) == 1
    assert np.all(Ey == 0.3) and np.all(Bz == 0.0)
    # B follows the new E_z within the step: dB_y/dt = d E_z at nodes 4, 5
    assert By[4] == pytest.approx(-DT * DT * 0.012 / DX, rel=1e-12)
    assert By[5] == pytest.approx(DT * DT * 0.012 / DX, rel=1e-12)
    assert np.count_nonzero(By) == 2


def test_drift_in_E_z_goes_along_y():
    """E_z = 0.5: v_y = +E_z / B_* = 0.05, j_y = (+1)(0.1)(0.05)/0.5 = 0.01
    for a positron at rest in cell 7."""
    s = _sim()
    _uniform(s, Ez=0.5)
    s.add_lepton(1, +1, 7.5, 0.0, 0.1)
    s.step(1)
    Jy, Jz = s.jperp()
    assert Jy[7] == pytest.approx(0.01, rel=1e-14)
    assert np.count_nonzero(Jy) == 1 and np.count_nonzero(Jz) == 0


@pytest.mark.parametrize("X,cells,shares", [(4.8, (4, 5), (0.7, 0.3)), (4.2, (3, 4), (0.3, 0.7)),
                                            (15.9, (15, 0), (0.6, 0.4))])
def test_cloud_shares_between_two_cells(X, cells, shares):
    """The unit cloud [X - 1/2, X + 1/2] on the cells it overlaps (periodic
    wrap at the top); the shares sum to the particle's whole current."""
    s = _sim()
    _uniform(s, Ey=0.3)
    s.add_lepton(1, -1, X, 0.0, 0.2)
    s.step(1)
    _, Jz = s.jperp()
    for c, f in zip(cells, shares):
        assert Jz[c] == pytest.approx(0.012 * f, rel=1e-12)
    assert Jz.sum() * DX == pytest.approx(0.2 * 0.03, rel=1e-12)


def test_sliding_along_a_tilted_field_line():
    """An electron with u = 3 (beta_h = 3 / sqrt 10) in B_y = 0.5,
    B_z = -0.2 and no E: v = beta_h (B_y, B_z) / B_*; deposited at its
    start-of-step position (cell 5 exactly), then dE_perp = -dt j_perp."""
    s = _sim()
    _uniform(s, By=0.5, Bz=-0.2)
    s.add_lepton(1, -1, 5.5, 3.0, 0.4)
    s.step(1)
    bh = 3.0 / math.sqrt(10.0)
    jy, jz = -0.4 * bh * 0.5 / BS / DX, -0.4 * bh * (-0.2) / BS / DX
    Jy, Jz = s.jperp()
    assert Jy[5] == pytest.approx(jy, rel=1e-14) and Jz[5] == pytest.approx(jz, rel=1e-14)
    assert np.count_nonzero(Jy) == 1 and np.count_nonzero(Jz) == 1
    Ey, Ez, _, _ = s.em()
    assert Ey[5] == pytest.approx(-DT * jy, rel=1e-14) and Ez[5] == pytest.approx(-DT * jz, rel=1e-14)


def test_a_pair_at_rest_carries_no_drift_current():
    """Both charges drift the same way, so equal weights at one place cancel
    exactly, and so do an electron and a proton (the drift is mass-free)."""
    for add in (lambda s: s.add_lepton(2, +1, 6.3, 0.0, 0.25), lambda s: s.add_proton(2, 6.3, 0.0, 0.25)):
        s = _sim(protons=1)
        _uniform(s, Ey=0.3, Ez=-0.7)
        s.add_lepton(1, -1, 6.3, 0.0, 0.25)
        add(s)
        s.step(1)
        Jy, Jz = s.jperp()
        assert np.abs(Jy).max() < 1e-17 and np.abs(Jz).max() < 1e-17
        Ey, Ez, _, _ = s.em()
        assert np.all(Ey == 0.3) and np.all(Ez == -0.7)


def test_conductor_images_and_the_cloud_below_the_star():
    """Surface gap: at X = 0.2 the cloud covers the image cell -1 (share 0.3,
    no current) and cell 0 (0.7), and E_y there is the linear value between
    the image -E_y[0] and E_y[0]: 0.3 (-E_y[0]) + 0.7 E_y[0] = 0.4 E_y[0]."""
    s = _sim(boundary=O.BC_SURFACE)
    nx = s.cfg["nx"]
    Ey = np.zeros(nx)
    Ey[0], Ey[1] = 0.3, 5.0
    s.set_em(Ey, np.zeros(nx), np.zeros(nx + 1), np.zeros(nx + 1))
    s.add_lepton(1, -1, 0.2, 0.0, 0.2)
    s.step(1)
    Jy, Jz = s.jperp()
    vz = -(0.4 * 0.3) / BS
    assert Jz[0] == pytest.approx(-0.2 * vz * 0.7 / DX, rel=1e-13)
    assert np.count_nonzero(Jz) == 1 and np.count_nonzero(Jy) == 0


def test_off_without_jperp_and_the_drift_scales_as_one_over_B_star():
    """jperp = 0 leaves the transverse fields to the virtual current alone;
    doubling b doubles B_* and halves the drift current."""
    s = O.Sim(nx=16, dx=DX, dt=DT, boundary=O.BC_PERIODIC, em=1, jperp=0, b=B_, lambda_hat=LAM)
    s.set_E(np.zeros(s.nnode))
    _uniform(s, Ey=0.3)
    s.add_lepton(1, -1, 4.5, 0.0, 0.2)
    s.step(1)
    assert np.all(s.em()[1] == 0.0)
    s2 = O.Sim(nx=16, dx=DX, dt=DT, boundary=O.BC_PERIODIC, em=1, jperp=1, b=2 * B_, lambda_hat=LAM)
    s2.set_E(np.zeros(s2.nnode))
    _uniform(s2, Ey=0.3)
    s2.add_lepton(1, -1, 4.5, 0.0, 0.2)
    s2.step(1)
    assert s2.jperp()[1][4] == pytest.approx(0.006, rel=1e-14)
