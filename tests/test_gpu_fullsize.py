"""The roofline workload at its full size, in the launch configuration the
bench times: Nx = 2^20 periodic cells, 200 e- + 200 e+ per cell (4.19e8
leptons), Maxwell-Juttner theta = 0.1, 1e-3 Langmuir seed, FP32 state, tile
256, 256 threads, the lean push.  The oracle cannot step 4e8 leptons, but it
can push any one of them: a fixed sample (ids divisible by 20000, about 1e4
per species) is pushed one step by the oracle from the GPU's own state and
field E^n, and must match the GPU's step to FP32 rounding.  Gauss's law,
which holds at any size, is checked on the whole gap."""
import numpy as np
import pytest

import bench
import oracle as O

pytestmark = pytest.mark.gpu

STRIDE = 20000


def test_config2_full_size_sampled_push_and_gauss():
    from paper_2608_21920_b300 import Gap
    cfg = dict(bench.WORKLOAD, nx=1 << 20, seed=0, gap_index=0)
    nx = cfg["nx"]
    g = Gap(cfg, precision="fp32", tile=256, threads=256, variant=0)
    try:
        g.step(3)
        E = g.field()
        before = [g.sample_particles(kind, STRIDE) for kind in (0, 1)]
        g.step(1)
        after = [g.sample_particles(kind, STRIDE) for kind in (0, 1)]
        d = g.diag(spectrum=False)
    finally:
        g.close()
    assert d["n_electrons"] + d["n_positrons"] == 2 * nx * cfg["ppc"]
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])

    o = O.Sim(nx=nx, boundary=O.BC_PERIODIC, dx=cfg["dx"], dt=cfg["dt"], init=O.INIT_EMPTY)
    o.set_E(E)
    for kind, q in ((0, -1), (1, 1)):
        b = before[kind]
        assert b["id"].size > 9000  # about 1e4 per species
        for i in range(b["id"].size):
            o.add_lepton(int(b["id"][i]), q, float(b["X"][i]), float(b["u"][i]), float(b["w"][i]))
    o.step(1)
    L = o.leptons()
    got = {k: np.concatenate([a[k] for a in after]) for k in ("id", "X", "u")}
    gi, oi = np.argsort(got["id"]), np.argsort(L["id"])
    assert np.array_equal(got["id"][gi], L["id"][oi])  # periodic: every sampled lepton is still there
    dX = got["X"][gi] - L["X"][oi]
    dX -= nx * np.round(dX / nx)
    du = got["u"][gi] - L["u"][oi]
    # FP32 offsets (2^-23 cells) and momenta; the kick of this step is ~1e-4,
    # the drift ~0.2 cells, so a wrong sign or term is far outside these
    assert np.abs(dX).max() < 2e-6
    assert np.abs(du).max() < 2e-6 * max(1.0, np.abs(L["u"]).max())
    moved = np.abs((L["X"][oi] - np.concatenate([b["X"] for b in before])[np.argsort(
        np.concatenate([b["id"] for b in before]))]))
    assert np.median(np.minimum(moved, nx - moved)) > 1e-3  # the leptons did move


def test_config2_full_size_window_field_parity():
    """E^{n+1} at full size, node by node: the leptons of four tiles (1024
    nodes) and of one tile of halo on each side are exported from the GPU
    (gap_tile_particles), pushed one step by the oracle from the GPU's own
    state and E^n, and the oracle's E^{n+1} = E^n + dt (j_m - J) on every
    node of the four tiles must match the GPU's.  The difference comes only
    from FP32 positions: each lepton's new offset lies within 2^-23 (grid) +
    2^-23 (rounding of the FP32 drift) of the FP64 one, and at most the ~400
    leptons whose clouds straddle a node move its charge, so per node
    |dE| <= 400 w0 2^-22 (w0 = 2.5e-4); the step's own change of E is ~1e-3."""
    from paper_2608_21920_b300 import Gap
    cfg = dict(bench.WORKLOAD, nx=1 << 20, seed=0, gap_index=0)
    nx, tile = cfg["nx"], 256
    t_lo, t_hi = 1000, 1004
    g = Gap(cfg, precision="fp32", tile=tile, threads=256, variant=0)
    try:
        g.step(3)
        E0 = g.field()
        lep = [g.tile_particles(kind, t_lo - 1, t_hi + 1) for kind in (0, 1)]
        c = g.diag(spectrum=False)["counters"]
        g.step(1)
        E1 = g.field()
    finally:
        g.close()
    assert c["spilled"] == 0
    o = O.Sim(nx=nx, boundary=O.BC_PERIODIC, dx=cfg["dx"], dt=cfg["dt"], init=O.INIT_EMPTY)
    o.set_E(E0)
    w0 = cfg["density"] * cfg["dx"] / cfg["ppc"] / 2
    for kind, q in ((0, -1), (1, 1)):
        L = lep[kind]
        assert L["id"].size > 6 * tile * cfg["ppc"] * 0.9
        assert np.allclose(L["w"], w0, rtol=1e-12)
        for i in range(L["id"].size):
            o.add_lepton(int(L["id"][i]), q, float(L["X"][i]), float(L["u"][i]), float(L["w"][i]))
    o.step(1)
    Eo = o.E()
    nodes = np.arange(t_lo * tile, t_hi * tile + 1)
    err = np.abs(E1[nodes] - Eo[nodes])
    dE = np.abs(Eo[nodes] - E0[nodes])
    assert err.max() <= 400 * w0 * 2.0 ** -22, err.max()
    assert np.median(dE) > 1e3 * 400 * w0 * 2.0 ** -22  # the step moved E far more than the bound
