"""Protons on the CUDA path (FP64 state) against the FP64 oracle: the Sect.
6.1 start (electrons everywhere, protons below H_gap, the linear ramp of E),
the proton push (kick by 1/m_ion, flux into the deferred Ampere step), and
the surface supply in both signs."""
import numpy as np
import pytest

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10
START = dict(nx=128, ppc=4, dx=0.1, dt=0.045, alpha=2.0, b=0.1, qed=1, lambda_hat=2e-4, rho_hat=10.0,
             rate_mult=5.0, init=O.INIT_GAP_PROTONS, boundary=O.BC_SURFACE, seed=3, protons=1)


def _protons_gpu(g, gap=0):
    p = g.particles(3, gap)
    order = np.argsort(p["id"], kind="stable")
    return {k: v[order] for k, v in p.items()}


def _split_oracle(o):
    L = o.leptons()
    order = np.argsort(L["id"], kind="stable")
    L = {k: v[order] for k, v in L.items()}
    e = {k: v[L["heavy"] == 0] for k, v in L.items()}
    p = {k: v[L["heavy"] == 1] for k, v in L.items()}
    return e, p


def _parity(cfg, checkpoints):
    g, o = P.make_pair(cfg, "fp64", tile=32)
    P.compare_field(g.field(), o.E(), RTOL64, "initial E (the ramp)")
    n_prev = 0
    for n in checkpoints:
        g.step(n - n_prev)
        o.step(n - n_prev)
        n_prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"step {n}")
        e_o, p_o = _split_oracle(o)
        P.compare_leptons(P.leptons_gpu(g), e_o, RTOL64, f"leptons step {n}")
        pg = _protons_gpu(g)
        pg["q"] = np.ones(pg["id"].size, np.int32)
        P.compare_leptons(pg, p_o, RTOL64, f"protons step {n}")
        assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    return g, o


def test_proton_start_parity():
    """The Sect. 6.1 start with QED: the ramp, then electrons, protons, E and
    counters at 1e-10 over 400 steps."""
    g, o = _parity(START, [1, 100, 400])
    _, p_o = _split_oracle(o)
    assert p_o["id"].size > 300 and np.abs(p_o["u"]).max() > 0
    g.close()


def test_negative_alpha_with_protons_parity():
    """alpha = -2 with a T = 0.3 atmosphere and protons: the surface draws
    electrons and protons; parity at 1e-10 over 600 steps."""
    cfg = dict(START, alpha=-2.0, qed=0, inject_theta=0.3)
    g, o = _parity(cfg, [50, 300, 600])
    c = o.counters()
    assert c["injected"] > 0 and c["absorbed"] > 0
    g.close()


def test_protons_under_a_cap_parity():
    """The cap bounds e+- and photons only (R28): the electrons merge, the
    protons are left alone; everything at 1e-10 against the oracle."""
    g, o = _parity(dict(START, cap=300), [1, 100, 400])
    assert o.counters()["merged"] > 0
    g.close()


@pytest.mark.parametrize("alpha,theta", [(2.0, 0.0), (-2.0, 0.3)])
def test_protons_fp32_state_track_oracle(alpha, theta):
    """FP32 state with protons (QED off, so that both sides take the same
    events): the protons' positions sit on the state's offset grid, so the
    Gauss law holds to round-off; e+-, protons and E follow the oracle
    within the FP32 bound of a short run (2e-4 relative, E 1e-3), and the
    surface supply within a few macro-particles."""
    cfg = dict(START, qed=0, alpha=alpha, inject_theta=theta)
    g, o = P.make_pair(cfg, "fp32", tile=32)
    d = g.diag(spectrum=False)
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    g.step(60)
    o.step(60)
    d = g.diag(spectrum=False)
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    Eg, Eo = g.field(), o.E()
    assert np.abs(Eg - Eo).max() <= 1e-3 * np.abs(Eo).max()
    e_o, p_o = _split_oracle(o)
    pg = _protons_gpu(g)
    assert abs(pg["id"].size - p_o["id"].size) <= 3
    common, ia, ib = np.intersect1d(pg["id"], p_o["id"], return_indices=True)
    assert common.size >= p_o["id"].size - 3
    assert np.abs(pg["X"][ia] - p_o["X"][ib]).max() <= 2e-4 * max(1.0, np.abs(p_o["X"]).max())
    assert abs(d["counters"]["injected"] - o.counters()["injected"]) <= 3
    g.close()
