"""Pins of the oracle's spectra (Sect. 6.4, Fig. 6: the pair plasma's
momentum distribution dn/d ln p over h in [0, H_gap] and the photon energy
spectrum) and of its return-flux tally (Sect. 6.5, Fig. 7: the pairs that
fall onto the star, by Lorentz factor), on hand-built loads whose bins and
weights are written down here."""
import math

import numpy as np
import pytest

import oracle as O

DX = 0.1


def _gap():
    # H_gap = 20 cells of the 64
    return O.Sim(nx=64, dx=DX, gap_length=20 * DX, boundary=O.BC_SURFACE, init=O.INIT_EMPTY)


def test_spectra_bin_the_gap_by_ln_p_and_ln_x():
    """Eight bins of ln p over [0, 8): a lepton with p = e^(k + 1/2) lands in
    bin k with its weight; p = 0 and p below e^0 land in bin 0, p above e^8
    in bin 7; leptons and photons at or above H_gap are left out; protons
    are not part of the pair plasma."""
    s = _gap()
    pid = iter(range(1, 1000))
    expect_e, expect_p, expect_ph = np.zeros(8), np.zeros(8), np.zeros(8)
    for k in range(8):
        w = 0.01 * (k + 1)
        s.add_lepton(next(pid), -1, 3.5 + k, math.exp(k + 0.5), w)         # e-, up
        s.add_lepton(next(pid), +1, 4.25 + k, -math.exp(k + 0.5), 2 * w)   # e+, down: |u|
        expect_e[k] += w
        expect_p[k] += 2 * w
        s.add_photon(next(pid), 2.5 + k, math.exp(k + 0.5), 3 * w, 1, 0, 1e30)
        expect_ph[k] += 3 * w
    s.add_lepton(next(pid), -1, 1.5, 0.0, 0.5)          # p = 0: first bin
    s.add_lepton(next(pid), -1, 1.5, 0.3, 0.25)         # ln p < 0: first bin
    s.add_lepton(next(pid), +1, 1.5, math.exp(9.0), 0.125)  # above the range: last bin
    expect_e[0] += 0.75
    expect_p[7] += 0.125
    s.add_lepton(next(pid), -1, 20.0, 5.0, 7.0)         # at H_gap: out
    s.add_lepton(next(pid), -1, 45.0, 5.0, 7.0)         # above: out
    s.add_photon(next(pid), 30.0, 5.0, 7.0, 1, 0, 1e30)  # above: out
    s.add_proton(next(pid), 5.5, 0.1, 7.0)             # protons: out
    lep, ph = s.spectra(8, 0.0, 8.0)
    assert np.allclose(lep[0], expect_e, rtol=1e-15, atol=0)
    assert np.allclose(lep[1], expect_p, rtol=1e-15, atol=0)
    assert np.allclose(ph, expect_ph, rtol=1e-15, atol=0)


def test_return_flux_tally_by_gamma():
    """Leptons just above the star moving down at gamma = 10^((i + 1/2)/8)
    (so beta c dt > their height) are absorbed in one step and tallied with
    their weight in bin i; one moving up, and a proton falling in, are not
    tallied; the tally matches the absorbed count and the ledger's w gamma."""
    s = _gap()
    rows = []
    pid = 1
    for i in (0, 3, 8, 20, 40, 63):
        g = 10 ** ((i + 0.5) / 8)
        if g < 1.6:
            g = 1.6  # beta >= 0.78: crosses h = 0 in one step from X = 0.2
        u = -math.sqrt(g * g - 1)
        w = 0.001 * (i + 1)
        s.add_lepton(pid, -1 if i % 2 else 1, 0.2, u, w)
        rows.append((int(math.floor(math.log(math.sqrt(1 + u * u)) / (math.log(10) / 8))), w, math.sqrt(1 + u * u)))
        pid += 1
    s.add_lepton(pid, -1, 0.2, 3.0, 1.0)        # moving up: stays
    s.add_proton(pid + 1, 0.1, -0.5, 1.0)       # a proton falling in: not a pair
    s.step(1)
    h = s.return_spectrum()
    expect = np.zeros(64)
    for b, w, _ in rows:
        expect[min(b, 63)] += w
    assert np.allclose(h, expect, rtol=1e-15, atol=0)
    c = s.counters()
    assert c["absorbed"] == len(rows) + 1  # the proton is absorbed too, but not tallied
    e_pairs = sum(w * g for _, w, g in rows)
    assert c["e_absorbed"] > e_pairs  # plus the proton's m_ion w gamma


def test_return_spectrum_of_a_discharge_accounts_for_every_absorbed_pair():
    """Over a short QED discharge with pairs falling back, the tally agrees
    with the energy ledger: every tallied weight carries at least its bin's
    lowest gamma, and the ledger's absorbed energy is the sum of w gamma."""
    s = O.Sim(nx=128, ppc=4, dx=0.1, dt=0.045, alpha=1.5, b=0.1, qed=1, lambda_hat=2e-4, rho_hat=10.0,
              rate_mult=5.0, init=O.INIT_COLD, boundary=O.BC_SURFACE, seed=3)
    s.step(900)
    h = s.return_spectrum()
    c = s.counters()
    assert c["absorbed"] > 0 and h.sum() > 0
    g_lo = 10 ** (np.arange(64) / 8)
    assert (h * g_lo).sum() <= c["e_absorbed"] * (1 + 1e-12)
