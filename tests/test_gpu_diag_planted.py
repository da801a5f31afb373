"""The CUDA path's diagnostic summary (gap_diag, Sect. 6.2 Fig. 5 and
Sect. 6.6) on the hand-built loads whose numbers the oracle is pinned to:
multiplicity by species and direction, the peak cell, <gamma^-3> at the peak,
the gap edge at a straddling cell, E's extrema over the gap nodes and the
spectrum's Parseval sum."""
import math

import numpy as np
import pytest

import test_oracle_diag as T

pytestmark = pytest.mark.gpu


def _gpu_load(precision):
    from paper_2608_21920_b300 import Gap
    # a cap far above the load keeps per-particle weights without merging
    g = Gap(dict(nx=64, dx=T.DX, gap_length=T.HC * T.DX, init=0, boundary=0, cap=1 << 20),
            precision=precision, tile=16)
    ids, X, u, w, q = [], [], [], [], []

    def lep(qq, XX, uu, ww):
        ids.append(len(ids) + 1); q.append(qq); X.append(XX); u.append(uu); w.append(ww)

    for _ in range(2):
        lep(-1, 7.5, math.sqrt(3.0), 0.05)
    lep(-1, 7.5, -math.sqrt(8.0), 0.03)
    lep(+1, 7.5, math.sqrt(15.0), 0.02)
    lep(+1, 7.5, -math.sqrt(3.0), 0.07)
    lep(+1, 19.5, 0.0, 0.01)
    lep(-1, 20.5, 0.0, 1.0)
    lep(-1, 3.0, 0.0, 0.04)
    ids, X, u, w, q = map(np.array, (ids, X, u, w, q))
    for kind, sign in ((0, -1), (1, +1)):
        m = q == sign
        g.add_particles(kind, ids[m].astype(np.uint64), X[m], u[m], w[m], np.full(m.sum(), 1e30))
    n = 3
    g.add_particles(2, np.arange(100, 100 + n, dtype=np.uint64) | np.uint64(1 << 63), np.full(n, 7.5),
                    np.full(n, 10.0), np.full(n, 5.0), np.full(n, 1e30), n0=np.zeros(n, np.int64),
                    direction=np.ones(n))
    return g


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_planted_cloud_summary(precision):
    g = _gpu_load(precision)
    d = g.diag(spectrum=False, moments=True)
    assert d["n_photons"] == 3
    # FP32 stores weights in units of w0/256 and offsets on a 2^-23 grid
    tol = 1e-12 if precision == "fp64" else 1e-2
    assert d["peak_cell"] == 7
    assert d["M_peak"] == pytest.approx(T.M7, rel=tol)
    assert d["M_avg"] == pytest.approx(T.M_AVG, rel=tol)
    assert np.allclose(d["M_split"], T.SPLIT7, rtol=tol, atol=0)
    assert d["g3_peak"] == pytest.approx(T.G3_7, rel=max(tol, 1e-6))
    dens = d["moments"]["dens"]
    assert dens[0, 0, 20] == pytest.approx(10.0, rel=tol)
    assert dens[0, 0, 2] == pytest.approx(0.2, rel=tol) and dens[0, 0, 3] == pytest.approx(0.2, rel=tol)
    g.close()


def test_extrema_and_parseval_on_the_gpu():
    from paper_2608_21920_b300 import Gap
    g = Gap(dict(nx=64, dx=T.DX, gap_length=T.HC * T.DX, init=0, boundary=0), precision="fp64", tile=16)
    E = np.zeros(g.nnode())
    E[4], E[20], E[21], E[40] = -3.0, 5.0, 100.0, -100.0
    g.set_field(E)
    d = g.diag()
    assert d["E_max"] == 5.0 and d["E_min"] == -3.0
    rng = np.random.default_rng(5)
    E = rng.normal(size=g.nnode())
    g.set_field(E)
    spec = g.diag()["spectrum"]
    assert spec.size == 17
    assert T._one_sided_sum(spec) == pytest.approx(float((E[:21] ** 2).sum()), rel=1e-12)
    g.close()
