"""The particles' transverse current (guiding-centre limit of the strong
field, option jperp with em) on the CUDA path against the FP64 oracle: the
hand-worked single-particle cases the oracle is pinned to, and discharges in
which E_z is driven by nothing else, at 1e-10 with identical event counters
(with the paper's set-up options, protons and a batch mixed with gaps
without it), replayed from CUDA graphs, and the FP32 state within its
rounding bound."""
import math

import numpy as np
import pytest

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10
# a cap far above the load keeps the particles' own weights (no merging)
PIN = dict(nx=16, dx=0.5, dt=0.05, boundary=O.BC_PERIODIC, em=1, jperp=1, b=0.2, lambda_hat=0.02, cap=1 << 20)


def _compare_em(g, o, rtol, what, gap=0):
    for name, a, b in zip(("E_y", "E_z", "B_y", "B_z"), g.em(gap), o.em()):
        if np.abs(b).max() == 0.0:
            assert np.abs(a).max() == 0.0, f"{what}: {name} should stay zero"
        else:
            P.compare_field(a, b, rtol, f"{what} {name}")


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("case", ["drift", "cloud", "tilted", "wrap", "star"])
def test_single_particle_cases_match_the_oracle(precision, rtol, case):
    """One particle in uniform fields, one step: the change of E_perp (and
    of B_perp through it) equals the oracle's, whose values are worked by
    hand in the oracle's pins."""
    from paper_2608_21920_b300 import Gap
    cfg = dict(PIN, boundary=O.BC_SURFACE) if case == "star" else dict(PIN)
    nx = cfg["nx"]
    nn = nx + 1 if case == "star" else nx
    X, u, q = {"drift": (4.5, 0.0, -1), "cloud": (4.8, 0.0, -1), "tilted": (5.5, 3.0, -1),
               "wrap": (15.9, 0.0, 1), "star": (0.2, 0.0, -1)}[case]
    Ey, Ez = np.full(nx, 0.3), np.full(nx, -0.2)
    By, Bz = np.full(nn, 0.5 if case == "tilted" else 0.0), np.full(nn, -0.2 if case == "tilted" else 0.0)
    if case == "star":
        Ey[:] = 0.0
        Ey[0], Ey[1] = 0.3, 5.0
    w = 0.25
    g = Gap(P.gpu_params(cfg), precision=precision, tile=8)
    o = O.Sim(**cfg)
    for s in (g,):
        s.set_field(np.zeros(nn))
        s.set_em(Ey, Ez, By, Bz)
    o.set_E(np.zeros(nn))
    o.set_em(Ey, Ez, By, Bz)
    g.add_particles(0 if q < 0 else 1, np.array([1], np.uint64), np.array([X]), np.array([u]), np.array([w]),
                    np.array([1e30]))
    o.add_lepton(1, q, X, u, w)
    before = [f.copy() for f in o.em()]
    g.step(1)
    o.step(1)
    for name, a, b, b0 in zip(("E_y", "E_z", "B_y", "B_z"), g.em(), o.em(), before):
        d_o, d_g = b - b0, a - b0
        scale = np.abs(d_o).max()
        if scale == 0.0:
            assert np.abs(d_g).max() <= 1e-7 * max(1.0, np.abs(b0).max()), name
        else:
            assert np.abs(d_g - d_o).max() <= rtol * scale, (name, np.abs(d_g - d_o).max() / scale)
    g.close()


DISCHARGE_JP = dict(nx=256, ppc=4, dx=0.1, dt=0.045, boundary=O.BC_SURFACE, alpha=2.0, qed=1, b=0.1,
                    lambda_hat=1e-4, rho_hat=20.0, rate_mult=20.0, init=O.INIT_COLD, density=1.0, seed=3,
                    em=1, pml_cells=16, beta_y=3e-3, filter_passes=8, inject_theta=0.3, jperp=1)


def _parity(cfg, checkpoints, tile, graph_chunk=0, precision="fp64"):
    g, o = P.make_pair(cfg, precision, tile=tile)
    prev = 0
    for n in checkpoints:
        if graph_chunk:
            g.step(n - prev, graph_chunk=graph_chunk)
        else:
            g.step(n - prev)
        o.step(n - prev)
        prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"E_h step {n}")
        _compare_em(g, o, RTOL64, f"step {n}")
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), RTOL64, f"leptons step {n}")
        assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    return g, o


@pytest.mark.parametrize("graph_chunk", [0, 50])
def test_discharge_with_the_particle_current_parity(graph_chunk):
    """A QED discharge set-up (8-pass filter, T = 0.3 atmosphere, absorbing
    layer) with the frame moving along y: the virtual current has no z
    component, so E_z and B_y come from the particles alone; all fields,
    particles and counters at 1e-10, eager and from CUDA graphs."""
    g, o = _parity(DISCHARGE_JP, [1, 150, 400], tile=32, graph_chunk=graph_chunk)
    assert o.counters()["injected"] > 0
    Ey, Ez, By, Bz = o.em()
    assert np.abs(Ez).max() > 1e-9 * np.abs(Ey).max() > 0.0
    g.close()


def test_batch_mixed_with_gaps_without_it_parity():
    """Three gaps in one handle: with the particle current, with the frame's
    fields only, and without either; each against its own oracle."""
    from paper_2608_21920_b300 import Gap
    cfgs = [dict(DISCHARGE_JP, gap_index=0, filter_passes=0),
            dict(DISCHARGE_JP, gap_index=1, jperp=0, seed=4),
            dict(DISCHARGE_JP, gap_index=2, em=0, jperp=0, beta_y=0.0, pml_cells=0, seed=5)]
    batch = Gap([P.gpu_params(c) for c in cfgs], precision="fp64", tile=32)
    oracles = [O.Sim(**{k: v for k, v in c.items() if k in O.DEFAULTS}) for c in cfgs]
    batch.step(300)
    for i, (c, o) in enumerate(zip(cfgs, oracles)):
        o.step(300)
        P.compare_counters(batch.diag(i, spectrum=False)["counters"], o.counters(), f"gap {i}")
        P.compare_field(batch.field(i), o.E(), RTOL64, f"gap {i}")
        P.compare_leptons(P.leptons_gpu(batch, i), P.leptons_oracle(o), RTOL64, f"gap {i}")
        if c["em"]:
            _compare_em(batch, o, RTOL64, f"gap {i}", gap=i)
    assert np.abs(oracles[0].em()[1]).max() > 0.0 and np.abs(oracles[1].em()[1]).max() == 0.0
    batch.close()


def test_full_setup_with_protons_parity():
    """The paper's full set-up (start with protons, QED, 8-pass filter,
    T = 0.3 atmosphere, the frame at beta = 3e-3 with a 32-cell layer) and
    the particle current of e+- and protons: everything at 1e-10."""
    cfg = dict(nx=256, ppc=4, dx=0.1, dt=0.045, alpha=2.0, b=0.1, qed=1, lambda_hat=2e-4, rho_hat=10.0,
               rate_mult=5.0, init=O.INIT_GAP_PROTONS, boundary=O.BC_SURFACE, seed=3, protons=1, filter_passes=8,
               inject_theta=0.3, em=1, beta_y=3e-3, pml_cells=32, jperp=1)
    g, o = P.make_pair(cfg, "fp64", tile=32)
    prev = 0
    for n in (1, 400, 800):
        g.step(n - prev)
        o.step(n - prev)
        prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"E_h step {n}")
        _compare_em(g, o, RTOL64, f"step {n}")
    assert np.abs(o.em()[1]).max() > 0.0
    g.close()


def test_fp32_state_tracks_the_oracle():
    """Cold electrons accelerating from a surface with the frame moving along
    y (no QED): E_z exists only through the particles' drift in E_y.  The
    FP32 state's E_h, E_y and E_z within its rounding bound after 150 steps,
    Gauss's law to round-off."""
    cfg = dict(DISCHARGE_JP, qed=0, filter_passes=0, inject_theta=0.0, beta_y=0.05)
    g, o = P.make_pair(cfg, "fp32", tile=32)
    g.step(150)
    o.step(150)
    assert np.abs(g.field() - o.E()).max() <= 1e-3 * np.abs(o.E()).max()
    (Ey_g, Ez_g, _, _), (Ey_o, Ez_o, _, _) = g.em(), o.em()
    assert np.abs(Ez_o).max() > 0.0
    assert np.abs(Ey_g - Ey_o).max() <= 2e-3 * np.abs(Ey_o).max()
    assert np.abs(Ez_g - Ez_o).max() <= 1e-2 * np.abs(Ez_o).max()
    d = g.diag(spectrum=False)
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    g.close()


def test_options_are_checked():
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300._abi import GapError
    base = dict(nx=32, dx=0.1, dt=0.045, boundary=O.BC_SURFACE)
    for bad in (dict(jperp=1), dict(em=1, jperp=2), dict(em=1, jperp=1, b=0.0), dict(em=1, jperp=1, lambda_hat=0.0)):
        with pytest.raises(GapError):
            Gap(P.gpu_params(dict(base, **bad)), precision="fp64", tile=16)
