"""The merge's ln gamma bin floor(ln gamma / width) (R20) is taken from an
FP32 evaluation where that lies more than 1e-3 of a bin from a bin edge, and
from FP64 otherwise, so that the groups are those of the FP64 definition.
This checks the margin's premise without a GPU: over FP32 momenta of both
signs from 1e-4 to 1e6, including momenta placed on bin edges, and every
merge level (width 0.1 2^L, L = 0..7), the FP32 evaluation (IEEE single
precision: u^2, 1 + u^2, square root, logarithm, times the rounded
1/width) stays within 1e-4 of a bin of the FP64 one, and wherever the fast
path is taken its bin is the FP64 bin."""
import numpy as np
import pytest

BINS = 256


def _momenta():
    rng = np.random.default_rng(5)
    mag = 10.0 ** rng.uniform(-4, 6, 200000)
    u = (mag * np.where(rng.random(mag.size) < 0.5, -1.0, 1.0)).astype(np.float32)
    return u


def _edge_momenta(width):
    # u whose ln gamma sits on (or within rounding of) a bin edge
    b = np.arange(1, 200)
    with np.errstate(over="ignore"):
        g = np.exp(b * width)
        u = np.sqrt((g - 1.0) * (g + 1.0))
    u = u[np.isfinite(u) & (u < 3e38)].astype(np.float32)
    return np.concatenate([u, np.nextafter(u, np.float32(0)), np.nextafter(u, np.float32(np.inf)), -u])


@pytest.mark.parametrize("level", range(8))
def test_fp32_bin_within_margin_of_fp64(level):
    width = 0.1 * 2 ** level
    winv_f = np.float32(1.0 / width)
    u = np.concatenate([_momenta(), _edge_momenta(width)])
    with np.errstate(over="ignore"):
        uf = u.astype(np.float32)
        tf = np.log(np.sqrt(np.float32(1.0) + uf * uf, dtype=np.float32), dtype=np.float32) * winv_f
    ud = u.astype(np.float64)
    t64 = np.log(np.sqrt(1.0 + ud * ud)) / width
    ok = np.isfinite(tf) & (t64 < BINS - 1)
    assert np.max(np.abs(tf[ok].astype(np.float64) - t64[ok])) < 1e-4
    # where the kernel takes the FP32 bin, it is the FP64 bin
    tf, t64 = tf[ok], t64[ok]
    bf = np.floor(tf)
    fast = (tf - bf > 1e-3) & (bf + 1 - tf > 1e-3) & (tf < BINS - 1)
    b64 = np.clip(np.floor(t64), 0, BINS - 1)
    assert fast.sum() > 0.5 * fast.size  # (momenta below ~1e-2 sit within 1e-3 of the edge 0)
    assert np.array_equal(bf[fast], b64[fast])
