"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 path: particle state and E within 1e-10 relative, identical QED event
counts.  FP32 path: within the FP32 error bound stated per test, exact Gauss
law (integer charge deposit)."""
import math

import numpy as np
import pytest

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10


def _step_both(g, o, n):
    g.step(n)
    o.step(n)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_free_acceleration(precision):
    cfg = dict(nx=512, boundary=O.BC_PERIODIC, dx=0.1, dt=0.045, ppc=1, density=1e-20)
    g, o = P.make_pair(cfg, precision)
    E0 = -0.5
    g.set_field(np.full(512, E0))
    o.set_E(np.full(512, E0))
    w = 1e-20 * 0.1
    g.add_particles(0, [1], [10.0], [0.0], [w], [1e30])
    o.add_lepton(1, -1, 10.0, 0.0, w)
    _step_both(g, o, 400)
    a, b = P.leptons_gpu(g), P.leptons_oracle(o)
    tol = RTOL64 if precision == "fp64" else 2e-6
    P.compare_leptons(a, b, tol, "free acceleration")
    assert a["u"][0] == pytest.approx(0.5 * 400 * 0.045, rel=1e-13 if precision == "fp64" else 2e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_deposit_two_nodes(precision):
    cfg = dict(nx=8, boundary=O.BC_PERIODIC, dx=0.1, dt=0.045, ppc=1, density=10.0)
    g, o = P.make_pair(cfg, precision)
    g.set_field(np.zeros(8))
    v = 0.4 * 0.1 / 0.045
    u = v / math.sqrt(1 - v * v)
    w = 1.0  # = w0 (density dx / ppc): exact in the FP32 weight units
    g.add_particles(1, [1], [3.3], [u], [w], [1e30])
    o.add_lepton(1, +1, 3.3, u, w)
    _step_both(g, o, 1)
    Eg, Eo = g.field(), o.E()
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.allclose(Eg, Eo, atol=tol)
    assert Eg[3] == pytest.approx(-0.2, abs=tol) and Eg[4] == pytest.approx(-0.2, abs=tol)


def _parity_run(cfg, checkpoints, precision="fp64", **kw):
    period = cfg["nx"] if cfg.get("boundary") == O.BC_PERIODIC else None
    g, o = P.make_pair(cfg, precision, **kw)
    P.compare_field(g.field(), o.E(), RTOL64, "initial E")
    n_prev = 0
    for n in checkpoints:
        _step_both(g, o, n - n_prev)
        n_prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"step {n}")
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), RTOL64, f"step {n}", period)
    return g, o


def test_config1_parity_first_200_steps():
    """Config 1 (cold electrons, alpha = 1.5, surface injection, QED on):
    E and particle state to 1e-10, identical event counts, over 200 steps."""
    g, o = _parity_run(P.CONFIG1, [1, 10, 50, 100, 150, 200], tile=64)
    c = o.counters()
    assert c["injected"] > 0 and c["emit_events"] > 0 and c["escaped"] > 0


def test_discharge_parity_with_pairs():
    """Small surface discharge through photon emission, conversion and pair
    creation: parity over 700 steps."""
    g, o = _parity_run(P.SMALL_DISCHARGE, [100, 300, 500, 600, 700], tile=32)
    c = o.counters()
    assert c["pairs"] > 0 and c["photons"] > 0


@pytest.mark.parametrize("tile", [8, 32, 256])
def test_thermal_pairs_periodic_parity(tile):
    _parity_run(P.THERMAL_PAIRS, [1, 20, 60], tile=tile)


@pytest.mark.parametrize("tile", [8, 16, 64])
def test_ragged_tiles_surface(tile):
    cfg = dict(P.SMALL_DISCHARGE, nx=133, qed=0)
    _parity_run(cfg, [37, 150], tile=tile)


def test_fp32_state_tracks_oracle():
    """FP32 offsets and momenta: relative deviation grows like eps_32 x steps
    (1.2e-7 per step); the bound here is 2e-4 after 60 steps of a thermal
    plasma, and the Gauss law holds exactly (integer charge deposit)."""
    g, o = P.make_pair(P.THERMAL_PAIRS, "fp32", tile=32)
    _step_both(g, o, 60)
    a, b = P.leptons_gpu(g), P.leptons_oracle(o)
    dev = P.compare_leptons(a, b, 2e-4, "fp32 thermal", period=P.THERMAL_PAIRS["nx"])
    assert dev["X"] > 0  # genuinely a different precision
    Eg, Eo = g.field(), o.E()
    assert np.abs(Eg - Eo).max() <= 1e-3 * np.abs(Eo).max()
    d = g.diag(spectrum=False)
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
def test_fp32_push_variants_are_bit_identical(variant):
    """Every launch variant of the FP32 push (vector width, occupancy, TMA
    bulk-copy pipeline) performs the same arithmetic: states and E agree
    bit for bit with variant 0, on a periodic and on a surface gap."""
    from paper_2608_21920_b300 import Gap
    for cfg, tile in ((P.THERMAL_PAIRS, 32), (dict(P.SMALL_DISCHARGE, qed=0, nx=300), 64)):
        ref = Gap(P.gpu_params(cfg), precision="fp32", tile=tile, variant=0)
        alt = Gap(P.gpu_params(cfg), precision="fp32", tile=tile, variant=variant)
        ref.step(70)
        alt.step(70)
        assert np.array_equal(ref.field(), alt.field())
        a, b = P.leptons_gpu(ref), P.leptons_gpu(alt)
        assert np.array_equal(a["id"], b["id"])
        assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["u"], b["u"])
        assert ref.diag(spectrum=False)["counters"]["injected"] == alt.diag(spectrum=False)["counters"]["injected"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gauss_law_discharge(precision):
    g, o = P.make_pair(P.SMALL_DISCHARGE, precision, tile=32)
    g.step(800)
    d = g.diag(spectrum=False)
    assert d["counters"]["pairs"] > 0
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])


def test_diagnostics_match_oracle():
    g, o = P.make_pair(P.SMALL_DISCHARGE, "fp64", tile=32)
    _step_both(g, o, 450)
    d = g.diag(spectrum=True, moments=True)
    od = o.diag()
    om = o.moments()
    m = d["moments"]
    assert np.allclose(m["dens"], om["dens"], rtol=1e-9, atol=1e-12)
    assert np.allclose(m["g3w"], om["g3w"], rtol=1e-9, atol=1e-300)
    assert np.allclose(m["charge"], om["charge"], rtol=1e-9, atol=1e-12)
    assert d["M_peak"] == pytest.approx(od["M_peak"], rel=1e-9)
    assert d["M_avg"] == pytest.approx(od["M_avg"], rel=1e-9)
    assert d["peak_cell"] == od["peak_cell"]
    assert d["g3_peak"] == pytest.approx(od["g3_peak"], rel=1e-9)
    assert d["E_min"] == pytest.approx(od["E_min"], rel=1e-10) and d["E_max"] == pytest.approx(od["E_max"], abs=1e-10)
    assert np.allclose(d["spectrum"], od["spectrum"], rtol=1e-8, atol=1e-12 * od["spectrum"].max())
    r, emax = o.gauss_residual()
    assert d["gauss_residual"] <= 1e-12 * max(emax, 1.0) and r <= 1e-12 * max(emax, 1.0)
    # photons
    pg, po = g.particles(2), o.photons()
    assert pg["id"].size == po["id"].size
    i, j = np.argsort(pg["id"]), np.argsort(po["id"])
    assert np.array_equal(pg["id"][i], po["id"][j])
    assert np.allclose(pg["X"][i], po["X"][j], rtol=1e-12)
    assert np.allclose(pg["x"][i], po["x"][j], rtol=1e-10)
    assert np.allclose(pg["tau_acc"][i], po["tau_acc"][j], rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_spectrum_inverse_matches_oracle(precision, tol):
    """The emission sampler's inverse CDF of the classical curvature
    spectrum against the oracle's (independent quadrature and root finder)."""
    import torch
    g, _ = P.make_pair(dict(nx=16, ppc=1, qed=1), precision)
    U = np.concatenate([np.logspace(-16, -1, 60), np.linspace(0.05, 0.95, 60),
                        1 - np.logspace(-1, -7, 40)])
    xi = g.spectrum_inverse(torch.tensor(U)).cpu().numpy()
    ref = np.array([O.spec_inverse(u) for u in U])
    # relative in xi, or absolute where xi is far below the photon threshold
    err = np.abs(xi - ref) / np.maximum(ref, 1e-6)
    assert err.max() <= tol, (U[err.argmax()], xi[err.argmax()], ref[err.argmax()])


def test_photon_conversion_parity():
    cfg = dict(nx=512, boundary=O.BC_SURFACE, qed=1, b=0.1, lambda_hat=1e-4, rho_hat=20.0,
               rate_mult=10.0, dx=0.1, dt=0.045, gap_length=51.2, ppc=1, density=1e-6)
    g, o = P.make_pair(cfg, "fp64", tile=64)
    N = 400
    ids = np.arange(1, N + 1, dtype=np.uint64)
    ts = np.array([-math.log(O.uniform(5, int(i), 0, O.CH_BW_TAU, 0)) for i in ids])
    x = 30.0 + np.arange(N) % 50
    X = 1.0 + (np.arange(N) % 7) * 0.3
    dirs = np.where(np.arange(N) % 3 == 0, -1, 1)
    w = np.full(N, 1e-7)
    g.add_particles(2, ids, X, x, w, ts, n0=np.zeros(N, np.int64), direction=dirs)
    for i in range(N):
        o.add_photon(int(ids[i]), X[i], x[i], w[i], int(dirs[i]), 0, ts[i])
    for n in (50, 150, 250):
        _step_both(g, o, n - g.steps_done)
        cg, co = g.diag(spectrum=False)["counters"], o.counters()
        assert cg["pairs"] == co["pairs"] and cg["photons_escaped"] == co["photons_escaped"]
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), RTOL64, f"pairs step {n}")
    assert o.counters()["pairs"] > 50


def test_batched_gaps_match_single_runs():
    """Several independent gaps of different size in one handle evolve as
    when run alone (the batch is one launch per step)."""
    from paper_2608_21920_b300 import Gap
    cfgs = [dict(P.SMALL_DISCHARGE, nx=96, seed=1, gap_index=0),
            dict(P.SMALL_DISCHARGE, nx=160, alpha=-1.0, seed=2, gap_index=1),
            dict(P.THERMAL_PAIRS, nx=64, seed=3, gap_index=2)]
    batch = Gap([P.gpu_params(c) for c in cfgs], precision="fp64", tile=32)
    batch.step(400)
    for i, c in enumerate(cfgs):
        o = O.Sim(**{k: v for k, v in c.items() if k in O.DEFAULTS})
        o.step(400)
        P.compare_field(batch.field(i), o.E(), RTOL64, f"gap {i}")
        period = c["nx"] if c["boundary"] == O.BC_PERIODIC else None
        P.compare_leptons(P.leptons_gpu(batch, i), P.leptons_oracle(o), RTOL64, f"gap {i}", period)
        P.compare_counters(batch.diag(i, spectrum=False)["counters"], o.counters(), f"gap {i}")


def test_empty_gap_and_graph_replay():
    from paper_2608_21920_b300 import Gap
    import torch
    cfg = dict(nx=64, boundary=O.BC_SURFACE, alpha=2.0, ppc=4, density=1.0, init=O.INIT_EMPTY)
    g = Gap(P.gpu_params(cfg), precision="fp32", tile=16)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g.step(64, graph_chunk=16)
    torch.cuda.synchronize()
    o = O.Sim(**cfg)
    o.step(64)
    assert g.steps_done == 64
    d = g.diag(spectrum=False)
    # an empty gap with a surface fills with injected electrons; E follows
    assert d["counters"]["injected"] == o.counters()["injected"] > 0
    assert np.abs(g.field() - o.E()).max() <= 1e-5 * np.abs(o.E()).max()


def test_fp32_qed_two_pass_overflow_is_bit_identical():
    """The two-pass QED push with its list of deferred leptons cut to 4
    entries (2 tile movers, 2 emitters): the emitters and tile movers beyond
    them are found in the store by the overflow pass (an emitter by its node
    stored as -2 - k), and leptons, photons, E and the counters agree bit
    for bit with the push in place over a discharge that emits, converts and
    merges."""
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300 import _abi as A
    cfg = dict(P.SMALL_DISCHARGE, cap=450)
    ref = Gap(P.gpu_params(cfg), precision="fp32", tile=32, variant=2)
    alt = Gap(P.gpu_params(cfg), precision="fp32", tile=32, variant=0)
    A.check(A.lib().gap_defer_limit(alt.handle, 4), alt.handle, "gap_defer_limit")
    for n in (300, 400, 300):
        ref.step(n)
        alt.step(n)
        assert np.array_equal(ref.field(), alt.field())
        a, b = P.leptons_gpu(ref), P.leptons_gpu(alt)
        assert np.array_equal(a["id"], b["id"])
        for k in ("X", "u", "w", "tau"):
            assert np.array_equal(a[k], b[k]), k
        pa, pb = ref.particles(2), alt.particles(2)
        oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
        for k in ("id", "X", "x", "w", "tau_star"):
            assert np.array_equal(pa[k][oa], pb[k][ob]), k
        ca, cb = ref.diag(spectrum=False)["counters"], alt.diag(spectrum=False)["counters"]
        for k in P.COUNTER_KEYS:
            assert ca[k] == cb[k], k
    assert ca["pairs"] > 0 and ca["emit_events"] > 1000 and ca["merged"] > 0
    ref.close()
    alt.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("threads", [256, 128])
def test_fp32_qed_push_variants_are_bit_identical(variant, threads):
    """The FP32 QED push in two passes (variants 0 and 1: the quiet leptons
    streamed, the emitters and tile movers pushed by a second kernel from a
    list, Ampere after both) and in place (variant 2) performs the same
    arithmetic: over a discharge with emissions, photons, pairs and a cap
    that merges, leptons, photons, E and every counter agree bit for bit."""
    from paper_2608_21920_b300 import Gap
    cfg = dict(P.SMALL_DISCHARGE, cap=450)
    ref = Gap(P.gpu_params(cfg), precision="fp32", tile=32, variant=0, threads=threads)
    alt = Gap(P.gpu_params(cfg), precision="fp32", tile=32, variant=variant, threads=threads)
    for n in (300, 400, 300):
        ref.step(n)
        alt.step(n)
        assert np.array_equal(ref.field(), alt.field())
        a, b = P.leptons_gpu(ref), P.leptons_gpu(alt)
        assert np.array_equal(a["id"], b["id"])
        for k in ("X", "u", "w", "tau"):
            assert np.array_equal(a[k], b[k]), k
        pa, pb = ref.particles(2), alt.particles(2)
        oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
        for k in ("id", "X", "x", "w", "tau_star"):
            assert np.array_equal(pa[k][oa], pb[k][ob]), k
        ca, cb = ref.diag(spectrum=False)["counters"], alt.diag(spectrum=False)["counters"]
        for k in P.COUNTER_KEYS:  # the energy ledgers are atomic sums: equal up to their order
            assert ca[k] == cb[k], k
    assert ca["pairs"] > 0 and ca["emit_events"] > 0 and ca["merged"] > 0
    ref.close()
    alt.close()
