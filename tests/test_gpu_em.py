"""The transverse fields of the co-rotating frame (App. A, 1D reduction) on
the CUDA path against the FP64 oracle: E_y, E_z, B_y, B_z, the virtual
current's feedback on E_h and the particles, Gauss's law with the virtual
charge, and the absorbing layer at the top of a surface gap."""
import math

import numpy as np
import pytest

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10


def _compare_em(g, o, rtol, what):
    for name, a, b in zip(("E_y", "E_z", "B_y", "B_z"), g.em(), o.em()):
        if np.abs(b).max() == 0.0:
            assert np.abs(a).max() == 0.0, f"{what}: {name} should stay zero"
        else:
            P.compare_field(a, b, rtol, f"{what} {name}")


def _parity(cfg, checkpoints, tile, period=None, graph_chunk=0):
    g, o = P.make_pair(cfg, "fp64", tile=tile)
    n_prev = 0
    for n in checkpoints:
        if graph_chunk:
            g.step(n - n_prev, graph_chunk=graph_chunk)
        else:
            g.step(n - n_prev)
        o.step(n - n_prev)
        n_prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"E_h step {n}")
        _compare_em(g, o, RTOL64, f"step {n}")
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), RTOL64, f"leptons step {n}", period)
        r, _ = o.gauss_residual()
        assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"]), (d["gauss_residual"], r)
    return g, o


PAIRS_EM = dict(P.THERMAL_PAIRS, em=1, beta_y=0.2, beta_z=0.1)


@pytest.mark.parametrize("graph_chunk", [0, 25])
def test_em_pair_plasma_parity(graph_chunk):
    """A periodic thermal pair plasma with a large oblique beta (so that the
    virtual current visibly moves E_h): all fields and the particles at 1e-10,
    eager and from CUDA graphs."""
    g, o = _parity(PAIRS_EM, [1, 50, 150], tile=32, period=PAIRS_EM["nx"], graph_chunk=graph_chunk)
    Ey, Ez, By, Bz = o.em()
    assert np.abs(Ey).max() > 1e-4 and np.abs(Ez).max() > 1e-4 and np.abs(By).max() > 1e-4
    g.close()


DISCHARGE_EM = dict(nx=256, ppc=4, dx=0.1, dt=0.045, boundary=O.BC_SURFACE, alpha=2.0, qed=1, b=0.1,
                    lambda_hat=1e-4, rho_hat=20.0, rate_mult=20.0, init=O.INIT_COLD, density=1.0, seed=3,
                    em=1, pml_cells=16, beta_y=3e-3, filter_passes=8, inject_theta=0.3)


def test_em_discharge_with_layer_parity():
    """A QED discharge at a surface with the paper's set-up options (8-pass
    filter, T = 0.3 atmosphere) and an absorbing layer: everything at 1e-10,
    Gauss's law with the virtual charge outside the layer."""
    g, o = _parity(DISCHARGE_EM, [1, 150, 400], tile=32)
    assert np.abs(o.em()[0]).max() > 1e-4
    assert o.counters()["injected"] > 0
    g.close()


def test_em_vacuum_pulse_is_absorbed_by_the_layer():
    """A unit pulse set through the ABI runs up into the layer: the GPU and
    the oracle agree, and what the layer sends back is below 1e-5."""
    nx, pml = 400, 16
    cfg = dict(nx=nx, dx=0.1, dt=0.045, boundary=O.BC_SURFACE, em=1, pml_cells=pml)
    g, o = P.make_pair(cfg, "fp64", tile=64)
    dx, dt = 0.1, 0.045
    xc, xi = (np.arange(nx) + 0.5) * dx, np.arange(nx + 1) * dx
    f = lambda x: np.exp(-((x - 25.0) / 0.8) ** 2)  # noqa: E731
    fields = (f(xc + dt / 2), np.zeros(nx), np.zeros(nx + 1), f(xi))
    g.set_em(*fields)
    o.set_em(*fields)
    n = int((2 * (40 - 25) + 6) / dt)
    g.step(n)
    o.step(n)
    _compare_em(g, o, RTOL64, "pulse")
    ref = O.Sim(nx=1600, dx=dx, dt=dt, boundary=O.BC_SURFACE, em=1)
    xc2, xi2 = (np.arange(1600) + 0.5) * dx, np.arange(1601) * dx
    ref.set_em(f(xc2 + dt / 2), np.zeros(1600), np.zeros(1601), f(xi2))
    ref.step(n)
    Ey = g.em()[0]
    assert np.abs(Ey[: nx - pml] - ref.em()[0][: nx - pml]).max() < 1e-5
    g.close()


def test_em_fp32_state_tracks_oracle():
    """FP32 state (the lean push defers Ampere for the transverse fields): the
    fields within the FP32 bound of a short run of a thermal plasma, Gauss's
    law with the virtual charge to round-off."""
    g, o = P.make_pair(PAIRS_EM, "fp32", tile=32)
    g.step(60)
    o.step(60)
    Eg, Eo = g.field(), o.E()
    assert np.abs(Eg - Eo).max() <= 1e-3 * np.abs(Eo).max()
    for a, b in zip(g.em(), o.em()):
        assert np.abs(a - b).max() <= 2e-3 * np.abs(b).max()
    d = g.diag(spectrum=False)
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    g.close()


@pytest.mark.parametrize("variant", [2, 4])
def test_em_fp32_push_variants_are_bit_identical(variant):
    from paper_2608_21920_b300 import Gap
    ref = Gap(P.gpu_params(PAIRS_EM), precision="fp32", tile=32, variant=0)
    alt = Gap(P.gpu_params(PAIRS_EM), precision="fp32", tile=32, variant=variant)
    ref.step(70)
    alt.step(70)
    assert np.array_equal(ref.field(), alt.field())
    for a, b in zip(ref.em(), alt.em()):
        assert np.array_equal(a, b)
    ref.close()
    alt.close()


def test_em_checkpoint_resumes():
    """The transverse fields travel with the checkpoint.  FP64 state: the
    deferred flux is summed by double atomics, whose order varies between
    runs, so two runs agree to rounding (each tracks the oracle to 1e-10
    here), not bit for bit."""
    from paper_2608_21920_b300 import Gap
    cfg = P.gpu_params(DISCHARGE_EM)
    a = Gap(cfg, precision="fp64", tile=32)
    a.step(100)
    state = a.save()
    a.step(50)
    b = Gap(cfg, precision="fp64", tile=32)
    b.load(state)
    b.step(50)
    P.compare_field(b.field(), a.field(), 1e-9, "E_h after resume")
    for name, x, y in zip(("E_y", "E_z", "B_y", "B_z"), b.em(), a.em()):
        if np.abs(y).max() > 0:
            P.compare_field(x, y, 1e-9, f"{name} after resume")
    assert np.abs(a.em()[3]).max() > 1e-4
    a.close()
    b.close()


def test_em_options_are_checked():
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300._abi import GapError
    base = dict(nx=64, dx=0.1, dt=0.045, boundary=O.BC_SURFACE)
    for bad in (dict(beta_y=0.1), dict(pml_cells=8), dict(em=1, beta_y=0.8, beta_z=0.8),
                dict(em=1, beta_y=math.nan), dict(em=1, pml_cells=40), dict(em=2),
                dict(em=1, pml_cells=8, pml_sigma=-1.0), dict(em=1, pml_cells=8, boundary=O.BC_PERIODIC)):
        with pytest.raises(GapError):
            Gap(P.gpu_params(dict(base, **bad)), precision="fp64", tile=16)
    g = Gap(P.gpu_params(base), precision="fp64", tile=16)
    with pytest.raises(GapError):
        g.em()
    g.close()


def test_em_batch_mixed_with_plain_gaps_parity():
    """A batch of four gaps: with and without the transverse fields, periodic
    and surface; each gap against its own oracle at 1e-10."""
    from paper_2608_21920_b300 import Gap
    cfgs = [dict(PAIRS_EM, gap_index=0), dict(P.THERMAL_PAIRS, gap_index=1, seed=1),
            dict(DISCHARGE_EM, gap_index=2, filter_passes=0), dict(DISCHARGE_EM, gap_index=3, em=0, beta_y=0.0,
                                                                   pml_cells=0)]
    batch = Gap([P.gpu_params(c) for c in cfgs], precision="fp64", tile=32)
    oracles = [O.Sim(**{k: v for k, v in c.items() if k in O.DEFAULTS}) for c in cfgs]
    batch.step(300)
    for i, (c, o) in enumerate(zip(cfgs, oracles)):
        o.step(300)
        P.compare_field(batch.field(i), o.E(), RTOL64, f"gap {i}")
        period = c["nx"] if c["boundary"] == O.BC_PERIODIC else None
        P.compare_leptons(P.leptons_gpu(batch, i), P.leptons_oracle(o), RTOL64, f"gap {i}", period)
        if c.get("em"):
            for name, a, b in zip(("E_y", "E_z", "B_y", "B_z"), batch.em(i), o.em()):
                if np.abs(b).max() > 0:
                    P.compare_field(a, b, RTOL64, f"gap {i} {name}")
    batch.close()


def test_em_under_a_cap_parity():
    """Merging under a macro-particle cap with the transverse fields (oblique
    beta): fields, particles and counters at 1e-10 over 900 steps."""
    cfg = dict(DISCHARGE_EM, filter_passes=0, inject_theta=0.0, beta_y=0.05, beta_z=0.03, cap=450)
    g, o = _parity(cfg, [300, 900], tile=32)
    assert o.counters()["merged"] > 0
    g.close()


def test_em_full_setup_parity():
    """The paper's full set-up (start with protons, QED, 8-pass filter,
    T = 0.3 atmosphere, beta = 3e-6 with a 32-cell layer), FP64: e+-,
    protons, all fields and counters at 1e-10."""
    cfg = dict(nx=256, ppc=4, dx=0.1, dt=0.045, alpha=2.0, b=0.1, qed=1, lambda_hat=2e-4, rho_hat=10.0,
               rate_mult=5.0, init=O.INIT_GAP_PROTONS, boundary=O.BC_SURFACE, seed=3, protons=1, filter_passes=8,
               inject_theta=0.3, em=1, beta_y=3e-6, pml_cells=32)
    g, o = P.make_pair(cfg, "fp64", tile=32)
    prev = 0
    for n in (1, 400, 1000):
        g.step(n - prev)
        o.step(n - prev)
        prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"E_h step {n}")
        _compare_em(g, o, RTOL64, f"step {n}")
        L = o.leptons()
        order = np.argsort(L["id"], kind="stable")
        L = {k: v[order] for k, v in L.items()}
        e_o = {k: v[L["heavy"] == 0] for k, v in L.items()}
        p_o = {k: v[L["heavy"] == 1] for k, v in L.items()}
        P.compare_leptons(P.leptons_gpu(g), e_o, RTOL64, f"e+- step {n}")
        pg = g.particles(3)
        order = np.argsort(pg["id"], kind="stable")
        pg = {k: v[order] for k, v in pg.items()}
        pg["q"] = np.ones(pg["id"].size, np.int32)
        P.compare_leptons(pg, p_o, RTOL64, f"protons step {n}")
        assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_em_discharge_statements_of_sect_6_6(precision):
    """The three Sect. 6.6 statements the oracle checks on config 1 at
    beta = 3e-6, measured on the CUDA path's own fields: oscillations
    delta E_h / E_rot ~ 1e-2, |E_h(k)|^2 ~ k^-2, E_y ~ 1e-6 E_h."""
    from paper_2608_21920_b300 import Gap
    cfg = dict(P.CONFIG1, em=1, beta_y=3e-6, pml_cells=32)
    g = Gap(P.gpu_params(cfg), precision=precision, tile=64)
    Hc = int(0.8 * cfg["nx"])
    E_rot = 0.8 * cfg["nx"] * cfg["dx"]
    ratios, spec, osc = [], [], []
    w = np.hanning(Hc)
    for blk in range(40):
        g.step(100)
        E, Ey = g.field()[:Hc], g.em()[0][:Hc]
        ratios.append(np.abs(Ey).max() / np.abs(E).max())
        osc.append(np.abs((E - np.convolve(E, np.ones(16) / 16, mode="same"))[16:-16]).max() / E_rot)
        if blk >= 20:
            spec.append(np.abs(np.fft.rfft((E - E.mean()) * w)) ** 2)
    assert g.diag(spectrum=False)["counters"]["pairs"] > 1000
    S = np.mean(spec, axis=0)
    k = np.arange(S.size)
    band = (k >= 8) & (k <= 150)
    slope = np.polyfit(np.log(k[band]), np.log(S[band]), 1)[0]
    assert -2.7 < slope < -1.7, slope
    assert 1e-7 < np.median(ratios) < 1e-5, np.median(ratios)
    assert 1e-3 < max(osc) < 1e-1, max(osc)
    g.close()
