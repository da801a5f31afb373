"""The merge's spread D (weight-conserving merge of leptons under the cap):
the oracle sums D = sum w 2 sinh^2((asinh u - eta)/2) with the centre's
rapidity eta = ln(S+/S-)/2; the CUDA merge sums the same quantity written as
sum w (e - E)^2/(2 e E), e = gamma + u = exp(asinh u), E = exp(eta) =
sqrt(S+/S-), which needs no asinh or sinh per lepton.  Both are checked here
against the exact value of the definition, M^2 - W^2 = D (2W + D) with
M^2 = S+ S-, in extended precision, for warm, cold and nearly cold groups of
both directions (no GPU).  In nearly cold groups (D/W ~ 1e-14) the
difference asinh u - eta carries the rounding of two numbers of order
asinh u, ~1e-9 of D, and (e - E)^2 that of e and E alone, ~1e-11."""
import mpmath as mp
import numpy as np
import pytest

mp.mp.dps = 50


def _groups():
    rng = np.random.default_rng(11)
    out = []
    for centre, spread in ((0.3, 0.5), (-2.0, 0.1), (40.0, 1e-3), (-3e3, 1e-6), (1e5, 1e-7), (0.0, 1e-4)):
        n = int(rng.integers(3, 40))
        u = (centre + spread * abs(centre if centre else 1.0) * rng.standard_normal(n)).astype(np.float32)
        w = rng.integers(1, 1 << 12, n).astype(np.float64)
        out.append((u.astype(np.float64), w))
    return out


def _sums(u, w):
    big = np.sqrt(1.0 + u * u) + np.abs(u)
    e = np.where(u >= 0, big, 1.0 / big)
    sp = np.sum(w * e)
    sm = np.sum(w / e)
    return big, sp, sm


@pytest.mark.parametrize("k", range(6))
def test_spread_forms_agree_with_the_exact_value(k):
    u, w = _groups()[k]
    big, sp, sm = _sums(u, w)
    eta = 0.5 * np.log(sp / sm)
    d_sinh = np.sum(w * 2.0 * np.sinh(0.5 * (np.arcsinh(u) - eta)) ** 2)
    E = np.sqrt(sp / sm)
    d = np.where(u >= 0, big - E, 1.0 - E * big)
    d_exp = np.sum(w * d * d / big) / (2.0 * E)
    # exact: M^2 - W^2 = S+ S- - W^2 = D (2W + D)
    W = mp.fsum([mp.mpf(x) for x in w])
    Sp = mp.fsum([mp.mpf(wi) * (mp.sqrt(1 + mp.mpf(ui) ** 2) + mp.mpf(ui)) for ui, wi in zip(u, w)])
    Sm = mp.fsum([mp.mpf(wi) * (mp.sqrt(1 + mp.mpf(ui) ** 2) - mp.mpf(ui)) for ui, wi in zip(u, w)])
    D = float(mp.sqrt(Sp * Sm) - W)
    assert D >= 0.0
    assert abs(d_sinh - D) <= 5e-9 * D, (k, d_sinh, D)
    assert abs(d_exp - D) <= 2e-10 * D, (k, d_exp, D)
