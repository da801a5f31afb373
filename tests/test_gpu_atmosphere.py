"""The hot surface atmosphere (Sect. 6.1: atmospheric particles at
k_B T = 0.3 m_e c^2) on the CUDA path against the FP64 oracle: injected
electrons carry |u| of a 1D Maxwell-Juttner draw keyed by (id, step), so the
two sides hold the same electrons with the same momenta, and the energy
ledger credits w gamma."""
import numpy as np
import pytest

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10
LEDGER_KEYS = ("e_injected", "e_absorbed", "e_escaped", "work_jm", "e_radiated")

HOT = dict(P.SMALL_DISCHARGE, inject_theta=0.3)


def _compare_ledgers(cg, co, rtol, what):
    for k in LEDGER_KEYS:
        scale = max(abs(co[k]), 1e-300)
        assert abs(cg[k] - co[k]) <= rtol * scale + 1e-300, f"{what}: {k}: gpu {cg[k]} oracle {co[k]}"


def test_hot_atmosphere_discharge_parity():
    """A QED surface discharge fed by a T = 0.3 atmosphere: particle state and
    E to 1e-10, identical event counts and energy ledgers, over 700 steps."""
    g, o = P.make_pair(HOT, "fp64", tile=32)
    n_prev = 0
    for n in (1, 50, 200, 500, 700):
        g.step(n - n_prev)
        o.step(n - n_prev)
        n_prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        _compare_ledgers(d["counters"], o.counters(), 1e-10, f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"step {n}")
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), RTOL64, f"step {n}")
    c = o.counters()
    assert c["injected"] > 0 and c["pairs"] > 0 and c["load_overflow"] == 0
    g.close()


@pytest.mark.parametrize("precision,rtol,xtol", [("fp64", 1e-13, 1e-15), ("fp32", 1e-7, 2.5e-7)])
def test_first_injection_momenta(precision, rtol, xtol):
    """The first injection from an empty gap (cell-0 deficit dx on both sides):
    the same ids, X in (0, 1/2], u > 0 equal to the oracle's to the state's
    rounding, and the ledger's w gamma sum."""
    cfg = dict(nx=64, ppc=256, kmax_inject=512, boundary=O.BC_SURFACE, init=O.INIT_EMPTY,
               dx=0.1, dt=0.045, seed=7, inject_theta=0.3)
    g, o = P.make_pair(cfg, precision, tile=16, lepton_capacity=1 << 16)
    g.step(1)
    o.step(1)
    a, b = P.leptons_gpu(g), P.leptons_oracle(o)
    assert a["id"].size == b["id"].size > 200
    assert np.array_equal(a["id"], b["id"])
    assert np.all(a["u"] > 0)
    assert np.allclose(a["u"], b["u"], rtol=rtol, atol=0)
    assert np.abs(a["X"] - b["X"]).max() <= xtol  # offsets on a 2^-23 grid in FP32
    cg = g.diag(spectrum=False)["counters"]
    assert cg["injected"] == o.counters()["injected"]
    assert cg["e_injected"] == pytest.approx(np.sum(a["w"] * np.sqrt(1 + a["u"] ** 2)), rel=1e-12)
    g.close()


def test_hot_atmosphere_fp32_gauss():
    """FP32 state with a hot atmosphere and the lean push (QED off): injection
    keeps going and the Gauss law holds exactly (integer charge deposit)."""
    cfg = dict(HOT, qed=0, nx=1024, ppc=32)
    from paper_2608_21920_b300 import Gap
    g = Gap(P.gpu_params(cfg), precision="fp32", tile=256)
    g.step(200)
    d = g.diag(spectrum=False)
    assert d["counters"]["injected"] > 0
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    g.close()


def test_negative_alpha_parity():
    """alpha = -2 with a hot atmosphere: the injected electrons fall back onto
    the star and E grows as -alpha t in the bulk; parity to 1e-10 with
    identical injection and absorption counts over 1500 steps."""
    cfg = dict(HOT, alpha=-2.0)
    g, o = P.make_pair(cfg, "fp64", tile=16)
    n_prev = 0
    for n in (100, 600, 1500):
        g.step(n - n_prev)
        o.step(n - n_prev)
        n_prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        _compare_ledgers(d["counters"], o.counters(), 1e-10, f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"step {n}")
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), RTOL64, f"step {n}")
    c = o.counters()
    assert c["injected"] > 1000 and c["absorbed"] > 1000
    g.close()
