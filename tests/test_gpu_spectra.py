"""Spectra (Sect. 6.4, Fig. 6) and the return flux (Sect. 6.5, Fig. 7) on the
CUDA path: the hand-built load of the oracle's pins, and a QED discharge in
which the GPU's spectra and return tally match the oracle's."""
import math

import numpy as np
import pytest

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_spectra_of_a_planted_load(precision):
    from paper_2608_21920_b300 import Gap
    g = Gap(dict(nx=64, dx=0.1, gap_length=2.0, boundary=0, init=0, qed=1, rate_mult=0.0, cap=1 << 20),
            precision=precision, tile=16)
    expect = np.zeros((3, 8))
    e_rows, p_rows, ph_rows = [], [], []
    pid = 1
    for k in range(8):
        w = 0.01 * (k + 1)
        e_rows.append((pid, 3.5 + k, math.exp(k + 0.5), w)); expect[0, k] += w; pid += 1
        p_rows.append((pid, 4.25 + k, -math.exp(k + 0.5), 2 * w)); expect[1, k] += 2 * w; pid += 1
        ph_rows.append((pid, 2.5 + k, math.exp(k + 0.5), 3 * w)); expect[2, k] += 3 * w; pid += 1
    e_rows += [(pid, 1.5, 0.0, 0.5), (pid + 1, 1.5, 0.3, 0.25), (pid + 2, 20.0, 5.0, 7.0), (pid + 3, 45.0, 5.0, 7.0)]
    expect[0, 0] += 0.75
    p_rows.append((pid + 4, 1.5, math.exp(9.0), 0.125))
    expect[1, 7] += 0.125
    ph_rows.append((pid + 5, 30.0, 5.0, 7.0))
    for kind, rows in ((0, e_rows), (1, p_rows)):
        a = np.array(rows)
        g.add_particles(kind, a[:, 0].astype(np.uint64), a[:, 1], a[:, 2], a[:, 3], np.full(len(rows), 1e30))
    a = np.array(ph_rows)
    g.add_particles(2, a[:, 0].astype(np.uint64) | np.uint64(1 << 63), a[:, 1], a[:, 2], a[:, 3],
                    np.full(len(ph_rows), 1e30), n0=np.zeros(len(ph_rows), np.int64), direction=np.ones(len(ph_rows)))
    lep, ph = g.spectra(8, 0.0, 8.0)
    tol = 1e-14 if precision == "fp64" else 1e-2  # FP32 weights: multiples of w0/256
    assert np.allclose(lep, expect[:2], rtol=tol, atol=0)
    assert np.allclose(ph, expect[2], rtol=1e-14, atol=0)  # photons are FP64 in both states
    with pytest.raises(Exception):
        g.spectra(2000, 0.0, 8.0)
    g.close()


def test_discharge_spectra_and_return_flux_match_oracle_fp64():
    """The small surface discharge over 900 steps (pairs, photons, pairs
    falling back): the spectra of e-, e+ and photons in the gap and the
    return tally equal the oracle's bin by bin (1e-10 relative to the largest
    bin)."""
    g, o = P.make_pair(P.SMALL_DISCHARGE, "fp64", tile=32)
    g.step(900)
    o.step(900)
    P.compare_counters(g.diag(spectrum=False)["counters"], o.counters(), "step 900")
    for nbins, lo, hi in ((64, -4.0, 16.0), (200, 0.0, 12.0)):
        lg, pg = g.spectra(nbins, lo, hi)
        lo_, po = o.spectra(nbins, lo, hi)
        assert np.abs(lg - lo_).max() <= 1e-10 * lo_.max()
        assert np.abs(pg - po).max() <= 1e-10 * max(po.max(), 1e-300)
    assert po.sum() > 0 and lo_[1].sum() > 0  # photons and positrons present
    rg, ro = g.return_spectrum(), o.return_spectrum()
    assert ro.sum() > 0
    assert np.abs(rg - ro).max() <= 1e-10 * ro.max()
    g.close()


def test_discharge_return_flux_fp32_tracks_oracle():
    """FP32 state over the same discharge: the return tally's total weight and
    mean ln gamma within a few per cent of the oracle's (the FP32 run is not
    particle-by-particle comparable after the pairs start)."""
    g, o = P.make_pair(P.SMALL_DISCHARGE, "fp32", tile=32)
    g.step(900)
    o.step(900)
    rg, ro = g.return_spectrum(), o.return_spectrum()
    assert ro.sum() > 0
    assert abs(rg.sum() - ro.sum()) <= 0.05 * ro.sum()
    b = np.arange(64)
    assert abs((rg * b).sum() / rg.sum() - (ro * b).sum() / ro.sum()) <= 0.5  # bins of ln gamma
    g.close()
