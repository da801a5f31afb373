"""Pins of the oracle's diagnostic summary (Sect. 6.2, Fig. 5; Sect. 6.6).

The multiplicity is M = (n_e- + n_e+)/n_co per cell, split by species and by
direction of motion; the gap is the set of cells whose centre lies below
H_gap, and E's extrema and power spectrum are taken over the nodes at or
below H_gap.  These tests build loads by hand, with weights and momenta
chosen so that every expected number can be written down here, and check
`oracle.Sim.diag()` against those numbers.  A last test plants each of the
plausible slips (photons counted in M, the direction index swapped, the cell
that straddles H_gap counted as a gap cell, a wrong power of gamma) into the
oracle's summary and checks that the pins catch it.
"""
import math

import numpy as np
import pytest

import oracle as O

DX = 0.1
HC = 20.3  # H_gap in cells: cell 19 (centre 19.5) is in the gap, cell 20 (centre 20.5) is not


def _load():
    """The planted load (code units, n_co = 1, dx = 0.1):

    cell 7 (X = 7.5, whole cloud in the cell):
      e- up   : 2 x w = 0.05, u = +sqrt 3  (gamma 2)  -> density 1.0
      e- down : 1 x w = 0.03, u = -sqrt 8  (gamma 3)  -> 0.3
      e+ up   : 1 x w = 0.02, u = +sqrt 15 (gamma 4)  -> 0.2
      e+ down : 1 x w = 0.07, u = -sqrt 3  (gamma 2)  -> 0.7
      photons : 3 x w = 5 (must not count)
    cell 19 (in the gap): 1 e+ at rest, w = 0.01 (u = 0 counts as up) -> 0.1
    cell 20 (straddles H_gap, outside): 1 e- w = 1.0 -> 10
    node 3 (X = 3.0, cloud split between cells 2 and 3): 1 e- w = 0.04 at rest
    """
    s = O.Sim(nx=64, dx=DX, gap_length=HC * DX, boundary=O.BC_SURFACE, init=O.INIT_EMPTY)
    pid = iter(range(1, 100))
    for _ in range(2):
        s.add_lepton(next(pid), -1, 7.5, math.sqrt(3.0), 0.05)
    s.add_lepton(next(pid), -1, 7.5, -math.sqrt(8.0), 0.03)
    s.add_lepton(next(pid), +1, 7.5, math.sqrt(15.0), 0.02)
    s.add_lepton(next(pid), +1, 7.5, -math.sqrt(3.0), 0.07)
    for k in range(3):
        s.add_photon(next(pid), 7.5, 10.0, 5.0, +1, 0, 1e30)
    s.add_lepton(next(pid), +1, 19.5, 0.0, 0.01)
    s.add_lepton(next(pid), -1, 20.5, 0.0, 1.0)
    s.add_lepton(next(pid), -1, 3.0, 0.0, 0.04)
    return s


# Expected values, from the load above.
M7 = 1.0 + 0.3 + 0.2 + 0.7                                    # 2.2
SPLIT7 = np.array([[1.0, 0.3], [0.2, 0.7]])                    # [species e-, e+][up, down]
G3_7 = (0.10 / 8 + 0.03 / 27 + 0.02 / 64 + 0.07 / 8) / 0.22   # sum w gamma^-3 / sum w
M_AVG = (M7 + 0.1 + 0.2 + 0.2) / 20                           # 20 gap cells (0..19)


def _failures(d):
    """Deviations of a diagnostic summary from the planted load's numbers."""
    bad = []
    if not math.isclose(d["M_peak"], M7, rel_tol=1e-12):
        bad.append(("M_peak", d["M_peak"]))
    if d["peak_cell"] != 7:
        bad.append(("peak_cell", d["peak_cell"]))
    if not math.isclose(d["M_avg"], M_AVG, rel_tol=1e-12):
        bad.append(("M_avg", d["M_avg"]))
    if not np.allclose(np.asarray(d["M_split"]).reshape(2, 2), SPLIT7, rtol=1e-12, atol=0):
        bad.append(("M_split", d["M_split"]))
    if not math.isclose(d["g3_peak"], G3_7, rel_tol=1e-12):
        bad.append(("g3_peak", d["g3_peak"]))
    return bad


def test_planted_cloud_multiplicity_split_and_g3():
    s = _load()
    d = s.diag()
    assert _failures(d) == []


def test_moments_per_cell_of_the_planted_load():
    """The per-cell moments behind the summary: density by species and
    direction, charge, sum w and sum w gamma^-3; a cloud centred on node 3
    puts half its density into each of cells 2 and 3."""
    m = _load().moments()
    dens = m["dens"]
    assert np.allclose(dens[:, :, 7], SPLIT7, rtol=1e-12, atol=0)
    assert dens[0, 0, 2] == pytest.approx(0.2, rel=1e-12) and dens[0, 0, 3] == pytest.approx(0.2, rel=1e-12)
    assert dens[0, 0, 20] == pytest.approx(10.0, rel=1e-12) and dens[1, 0, 19] == pytest.approx(0.1, rel=1e-12)
    # nothing anywhere else
    mask = np.ones(64, bool)
    mask[[2, 3, 7, 19, 20]] = False
    assert np.all(dens[:, :, mask] == 0.0)
    assert m["charge"][7] == pytest.approx(-(0.10 + 0.03) + (0.02 + 0.07), rel=1e-12)
    assert m["wsum"][7] == pytest.approx(0.22, rel=1e-12)
    assert m["g3w"][7] == pytest.approx(G3_7 * 0.22, rel=1e-12)


def test_cold_load_has_unit_multiplicity():
    """Cold electrons at n_co (Sect. 6.1 start without protons), 16 per cell
    at X = c + (j + 1/2)/16: M = 1 in every gap cell but cell 0, all of it e-
    moving up (u = 0 counts as up), <gamma^-3> = 1.  The clouds of the eight
    electrons with X < 1/2 reach below the conductor at h = 0 by
    1/2 - (j + 1/2)/16, 2 cells of cloud in all, so cell 0 holds
    1 - 2/16 = 7/8 and the gap average is (19 + 7/8)/20."""
    s = O.Sim(nx=100, dx=DX, ppc=16, gap_length=HC * DX, init=O.INIT_COLD)
    m = s.moments()["dens"].sum(axis=(0, 1))
    assert m[0] == pytest.approx(7 / 8, rel=1e-12)
    assert np.allclose(m[1:99], 1.0, rtol=1e-12, atol=0)
    d = s.diag()
    assert d["M_peak"] == pytest.approx(1.0, rel=1e-12)
    assert d["M_avg"] == pytest.approx((19 + 7 / 8) / 20, rel=1e-12)
    assert np.allclose(np.asarray(d["M_split"]).reshape(2, 2), [[1.0, 0.0], [0.0, 0.0]], rtol=1e-12, atol=0)
    assert d["g3_peak"] == pytest.approx(1.0, rel=1e-15)
    assert 1 <= d["peak_cell"] < 20


def test_field_extrema_over_gap_nodes_only():
    """E's extrema are over nodes 0..floor(H_gap) (here 0..20): a spike on
    node 21 is outside, one on node 20 inside."""
    s = O.Sim(nx=64, dx=DX, gap_length=HC * DX, init=O.INIT_EMPTY)
    E = np.zeros(s.nnode)
    E[4], E[20], E[21], E[40] = -3.0, 5.0, 100.0, -100.0
    s.set_E(E)
    d = s.diag()
    assert d["E_max"] == 5.0 and d["E_min"] == -3.0


def _one_sided_sum(spec):
    w = np.full(spec.size, 2.0)
    w[0] = w[-1] = 1.0
    return float((w * spec).sum())


def test_spectrum_parseval_and_brute_force_dft():
    """|E_k|^2 / P over the 21 gap nodes zero-padded to P = 32: with the
    one-sided weights (1, 2, ..., 2, 1) the bins sum to sum E_i^2
    (Parseval), and every bin equals the directly summed DFT."""
    s = O.Sim(nx=64, dx=DX, gap_length=HC * DX, init=O.INIT_EMPTY)
    rng = np.random.default_rng(5)
    E = rng.normal(size=s.nnode)
    s.set_E(E)
    spec = s.diag()["spectrum"]
    P = 32
    assert spec.size == P // 2 + 1
    Eg = E[:21]
    assert _one_sided_sum(spec) == pytest.approx(float((Eg ** 2).sum()), rel=1e-12)
    i = np.arange(21)
    for k in range(P // 2 + 1):
        re = sum(Eg[j] * math.cos(2 * math.pi * k * j / P) for j in i)
        im = sum(Eg[j] * math.sin(2 * math.pi * k * j / P) for j in i)
        assert spec[k] == pytest.approx((re * re + im * im) / P, rel=1e-10, abs=1e-14)


def _planted_diag(s, mistake):
    """The oracle's summary with one slip planted in its input or rule."""
    cfg = dict(s.cfg)
    mom = s.moments()
    E = s.E()
    if mistake == "photons":
        ph = s.photons()
        for X, w in zip(ph["X"], ph["w"]):
            mom["dens"][0, 0, int(math.floor(X))] += w / cfg["dx"]
        return O.diag_from_state(cfg, mom, E)
    if mistake == "direction":
        mom["dens"] = mom["dens"][:, ::-1, :].copy()
        return O.diag_from_state(cfg, mom, E)
    if mistake == "species":
        mom["dens"] = mom["dens"][::-1, :, :].copy()
        return O.diag_from_state(cfg, mom, E)
    if mistake == "gap_edge":
        # cells below H_gap by their left edge instead of their centre
        cfg["gap_length"] = (math.floor(HC) + 1.0) * cfg["dx"]
        return O.diag_from_state(cfg, mom, E)
    if mistake == "g3_power":
        # gamma^-2 in place of gamma^-3
        L = s.leptons()
        inside = np.floor(L["X"]) == 7
        g = np.sqrt(1.0 + L["u"][inside] ** 2)
        mom["g3w"][7] = float((L["w"][inside] / g ** 2).sum())
        return O.diag_from_state(cfg, mom, E)
    raise KeyError(mistake)


@pytest.mark.parametrize("mistake", ["photons", "direction", "species", "gap_edge", "g3_power"])
def test_planted_mistakes_fail_the_pins(mistake):
    s = _load()
    assert _failures(_planted_diag(s, mistake)) != []
