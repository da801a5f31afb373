"""The 8-pass binomial current filter (Sect. 6.1) on the CUDA path against the
FP64 oracle: smoothed Ampere, smoothed Gauss solve and residual, smoothed
merge correction, per-gap switching inside a batch, the halo across tiles
narrower than the filter and the chunk loop of tiles wider than one
shared-memory round."""
import numpy as np
import pytest

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10


def _parity(cfg, checkpoints, precision="fp64", **kw):
    period = cfg["nx"] if cfg.get("boundary") == O.BC_PERIODIC else None
    g, o = P.make_pair(cfg, precision, **kw)
    P.compare_field(g.field(), o.E(), RTOL64, "initial E")
    n_prev = 0
    for n in checkpoints:
        g.step(n - n_prev)
        o.step(n - n_prev)
        n_prev = n
        d = g.diag(spectrum=False)
        P.compare_counters(d["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), RTOL64, f"step {n}")
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), RTOL64, f"step {n}", period)
        r, _ = o.gauss_residual()
        assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"]) and r <= 1e-12 * max(1.0, d["E_abs_max"])
        work = d["counters"]["work_jm"]
        assert abs(work - o.counters()["work_jm"]) <= 1e-10 * max(abs(work), 1e-300)
    return g, o


def test_filtered_discharge_parity():
    """A QED surface discharge with 8 smoothing passes: state, E, counters,
    the work of j_m and the smoothed Gauss law, over 700 steps."""
    g, o = _parity(dict(P.SMALL_DISCHARGE, filter_passes=8), [1, 100, 300, 500, 700], tile=32)
    assert o.counters()["pairs"] > 0
    g.close()


@pytest.mark.parametrize("tile", [8, 64])
def test_filtered_thermal_periodic_parity(tile):
    """Periodic wrap of the halos; with 8-node tiles the 8-node halo reaches
    past the neighbouring tile.  The initial field is the smoothed charge's."""
    _parity(dict(P.THERMAL_PAIRS, filter_passes=8), [1, 20, 60], tile=tile)


@pytest.mark.parametrize("passes", [1, 3, 16])
def test_filtered_ragged_surface_parity(passes):
    cfg = dict(P.SMALL_DISCHARGE, nx=133, qed=0, filter_passes=passes)
    _parity(cfg, [37, 150], tile=16)


def test_filter_chunk_loop_on_wide_tiles():
    """Tiles of 2048 nodes are smoothed in two shared-memory rounds."""
    cfg = dict(P.THERMAL_PAIRS, nx=4096, ppc=4, filter_passes=8)
    _parity(cfg, [1, 15], tile=2048)


def test_filtered_merge_parity():
    """Merging under a cap with the filter: the re-centring correction is
    smoothed like the current; FP64 parity over 900 steps."""
    g, o = _parity(dict(P.SMALL_DISCHARGE, cap=450, filter_passes=8), [300, 600, 900], tile=32)
    assert o.counters()["merged"] > 0
    g.close()


def test_filter_is_per_gap_in_a_batch():
    """A batch mixing a filter gap and unfiltered gaps: each evolves as alone."""
    from paper_2608_21920_b300 import Gap
    cfgs = [dict(P.SMALL_DISCHARGE, nx=96, seed=1, gap_index=0, filter_passes=8),
            dict(P.SMALL_DISCHARGE, nx=160, alpha=-1.0, seed=2, gap_index=1),
            dict(P.THERMAL_PAIRS, nx=64, seed=3, gap_index=2, filter_passes=4)]
    batch = Gap([P.gpu_params(c) for c in cfgs], precision="fp64", tile=32)
    batch.step(400)
    for i, c in enumerate(cfgs):
        o = O.Sim(**{k: v for k, v in c.items() if k in O.DEFAULTS})
        o.step(400)
        P.compare_field(batch.field(i), o.E(), RTOL64, f"gap {i}")
        period = c["nx"] if c["boundary"] == O.BC_PERIODIC else None
        P.compare_leptons(P.leptons_gpu(batch, i), P.leptons_oracle(o), RTOL64, f"gap {i}", period)
        P.compare_counters(batch.diag(i, spectrum=False)["counters"], o.counters(), f"gap {i}")
    batch.close()


def test_filtered_fp32_tracks_oracle():
    """FP32 state with the filter (the generic push; QED off so that both
    sides take the same events): the smoothed Gauss law to round-off and the
    field within the FP32 bound of a short run."""
    cfg = dict(P.SMALL_DISCHARGE, qed=0, filter_passes=8)
    g, o = P.make_pair(cfg, "fp32", tile=32)
    g.step(300)
    o.step(300)
    d = g.diag(spectrum=False)
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    Eg, Eo = g.field(), o.E()
    assert np.abs(Eg - Eo).max() <= 1e-3 * np.abs(Eo).max()
    assert d["counters"]["injected"] > 0
    g.close()


def test_filtered_fp32_merge_keeps_smoothed_gauss():
    cfg = dict(P.SMALL_DISCHARGE, filter_passes=8, cap=450)
    g, _ = P.make_pair(cfg, "fp32", tile=32)
    g.step(900)
    d = g.diag(spectrum=False)
    assert d["counters"]["merged"] > 0
    assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
    g.close()


def test_filter_rejects_bad_pass_counts():
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300._abi import GapError
    for bad in (dict(filter_passes=17), dict(filter_passes=-1), dict(nx=16, filter_passes=8)):
        with pytest.raises(GapError):
            Gap(P.gpu_params(dict(P.SMALL_DISCHARGE, **bad)), precision="fp64")


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
def test_filtered_fp32_push_variants_are_bit_identical(variant):
    """The lean and bulk-copy (TMA) FP32 pushes defer Ampere to the filter
    the same way: states and E agree bit for bit with variant 0 (integer
    charge accumulators make the smoothed field order-free)."""
    from paper_2608_21920_b300 import Gap
    for cfg, tile in ((dict(P.THERMAL_PAIRS, filter_passes=8), 32),
                      (dict(P.SMALL_DISCHARGE, qed=0, nx=300, filter_passes=8), 64)):
        ref = Gap(P.gpu_params(cfg), precision="fp32", tile=tile, variant=0)
        alt = Gap(P.gpu_params(cfg), precision="fp32", tile=tile, variant=variant)
        ref.step(70)
        alt.step(70)
        assert np.array_equal(ref.field(), alt.field())
        a, b = P.leptons_gpu(ref), P.leptons_gpu(alt)
        assert np.array_equal(a["id"], b["id"])
        assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["u"], b["u"])
        d = alt.diag(spectrum=False)
        assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
        ref.close()
        alt.close()


@pytest.mark.parametrize("passes", [1, 16])
def test_integer_smoothing_of_fp32_flux(passes):
    """The FP32 state smooths its integer flux in integers (split words, no
    division until the end): the smoothed Gauss law to round-off, the field
    within the FP32 bound of the FP64 oracle, at 1 and at the maximum 16
    passes, on a periodic and on a surface gap."""
    for cfg in (dict(P.THERMAL_PAIRS, filter_passes=passes),
                dict(P.SMALL_DISCHARGE, qed=0, filter_passes=passes)):
        g, o = P.make_pair(cfg, "fp32", tile=32)
        g.step(60)
        o.step(60)
        d = g.diag(spectrum=False)
        assert d["gauss_residual"] <= 1e-12 * max(1.0, d["E_abs_max"])
        Eg, Eo = g.field(), o.E()
        assert np.abs(Eg - Eo).max() <= 1e-3 * np.abs(Eo).max()
        g.close()
