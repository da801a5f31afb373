"""The quantum photon spectrum option (qed_quantum) on the CUDA path: the
table inverse against the oracle's exact inverse, and one emission of each of
800 leptons at chi = 2 against the oracle's emissions from the same draws.

Tolerance: the table interpolates ln s = ln d / 3 over rows of ln chi (eight
per decade, cubic) and the survival over 256 panels of s (cubic Hermite,
panels crowded towards s = 0); its emulation against the exact inverse stays
below 2e-5 relative in xi for chi in [1e-6, 1e5], so the FP64 bound is 1e-4.
The FP32 evaluation adds float rounding of the survival (1e-7 absolute):
relative 1e-3 for draws U <= 0.999."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu

QCFG = dict(nx=64, boundary=O.BC_PERIODIC, qed=1, qed_quantum=1, lambda_hat=2e-4, rho_hat=100.0,
            rate_mult=1e-3, dx=0.1, dt=0.045, gap_length=6.4)


def _gap(precision="fp64"):
    from paper_2608_21920_b300 import Gap
    return Gap(P.gpu_params(QCFG), precision=precision, tile=16)


@pytest.mark.parametrize("precision,rtol,umax", [("fp64", 1e-4, 1.0 - 1e-9), ("fp32", 1e-3, 0.999)])
def test_qspectrum_inverse_matches_oracle(precision, rtol, umax):
    g = _gap(precision)
    rng = np.random.default_rng(3)
    chis = [1e-7, 3e-6, 0.013, 0.7, 5.3, 77.0, 1e4, 1e5]
    Us = np.concatenate([rng.random(12) * umax, [1e-9, 1e-3, 0.5, umax]])
    chi = np.repeat(chis, Us.size)
    U = np.tile(Us, len(chis))
    xi = g.qspectrum_inverse(torch.tensor(chi), torch.tensor(U), precision).cpu().numpy()
    ref = np.array([O.qspec_inverse(c, u) for c, u in zip(chi, U)])
    assert np.all((xi > 0) & (xi < 1))
    rel = np.abs(xi / ref - 1.0)
    assert rel.max() <= rtol, (rel.max(), chi[rel.argmax()], U[rel.argmax()])
    g.close()


def test_qspectrum_inverse_needs_a_quantum_gap():
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300._abi import GapError
    g = Gap(P.gpu_params(dict(QCFG, qed_quantum=0)), precision="fp64", tile=16)
    with pytest.raises(GapError):
        g.qspectrum_inverse(torch.tensor([1.0]), torch.tensor([0.5]))
    g.close()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-4), ("fp32", 2e-3)])
def test_quantum_emission_matches_oracle(precision, rtol):
    """tau = 0 makes every lepton emit once at the start of the step (a second
    event in the step is improbable: rate x dt ~ 3e-6); the recoil gives the
    photon's energy fraction xi = (gamma0 - gamma)/gamma0."""
    g0, N = 1000.0, 800
    u0 = math.sqrt(g0 * g0 - 1.0)
    gpu = _gap(precision)
    o = O.Sim(**{k: v for k, v in QCFG.items() if k in O.DEFAULTS})
    ids = np.arange(1, N + 1)
    gpu.add_particles(0, ids, np.full(N, 1.0), np.full(N, u0), np.full(N, 1e-30), np.zeros(N))
    for i in ids:
        o.add_lepton(int(i), -1, 1.0, u0, 1e-30, tau=0.0)
    gpu.step(1)
    o.step(1)
    a, b = P.leptons_gpu(gpu), P.leptons_oracle(o)
    assert np.array_equal(a["id"], b["id"])
    xa = (g0 - np.sqrt(1.0 + a["u"] ** 2)) / g0
    xb = (g0 - np.sqrt(1.0 + b["u"] ** 2)) / g0
    assert gpu.diag(spectrum=False)["counters"]["emit_events"] == o.counters()["emit_events"]
    big = xb > 1e-3  # softer photons leave gamma unchanged to the state's rounding
    assert big.sum() > N // 2
    rel = np.abs(xa[big] / xb[big] - 1.0)
    assert rel.max() <= rtol, rel.max()
    gpu.close()


def test_pair_split_matches_oracle():
    """The electron's share of a conversion: the table against the oracle's
    exact inverse.  Its emulation bounds the smaller share's relative error
    by 1.6e-5 for u = min(U, 1 - U) >= 1e-3 and 3.7e-3 down to u = 1e-6
    (chi <= 1e4); the float inversion adds 1e-6; below chi = 1e-3 the
    Gaussian limit holds to O(chi)."""
    g = _gap("fp64")
    cases = [(chi, U) for chi in (2e-3, 0.05, 1.0, 77.0, 1e3, 5e3)
             for U in (1e-6, 1e-5, 1e-4, 1e-3, 0.01, 0.2, 0.45, 0.5, 0.7, 0.999, 1 - 1e-5)]
    chi = np.array([c for c, _ in cases])
    U = np.array([u for _, u in cases])
    e = g.pair_split(torch.tensor(chi), torch.tensor(U)).cpu().numpy()
    ref = np.array([O.bw_split(c, u) for c, u in cases])
    u = np.minimum(U, 1 - U)
    small_gpu, small_ref = np.minimum(e, 1 - e), np.minimum(ref, 1 - ref)
    rel = np.abs(small_gpu / small_ref - 1.0)
    off = U != 0.5
    assert np.all((e[off] < 0.5) == (U[off] < 0.5))
    assert rel[u >= 1e-3].max() <= 1e-4, rel[u >= 1e-3].max()
    assert rel.max() <= 6e-3, rel.max()
    # Gaussian limit below the table
    for c in (2e-4, 5e-4):
        eg = g.pair_split(torch.tensor([c] * 3), torch.tensor([0.1, 0.3, 0.9])).cpu().numpy()
        er = np.array([O.bw_split(c, x) for x in (0.1, 0.3, 0.9)])
        assert np.all(np.abs(eg - er) <= 5e-3 * np.abs(er - 0.5))
    g.close()


def test_quantum_pair_creation_matches_oracle():
    """Photons converting in a gap with qed_quantum: the same pairs at the same
    steps, the shares from the same draws (table tolerance), energy x split
    exactly between the two."""
    cfg = dict(nx=512, boundary=O.BC_SURFACE, qed=1, qed_quantum=1, b=0.1, lambda_hat=1e-4, rho_hat=20.0,
               rate_mult=10.0, dx=0.1, dt=0.045, gap_length=51.2, ppc=1, density=1e-6)
    g, o = P.make_pair(cfg, "fp64", tile=64)
    N = 200
    ids = np.arange(1, N + 1, dtype=np.uint64)
    ts = np.array([-math.log(O.uniform(5, int(i), 0, O.CH_BW_TAU, 0)) for i in ids])
    x = 30.0 + np.arange(N) % 50
    X = 1.0 + (np.arange(N) % 7) * 0.3
    dirs = np.where(np.arange(N) % 3 == 0, -1, 1)
    w = np.full(N, 1e-7)
    g.add_particles(2, ids, X, x, w, ts, n0=np.zeros(N, np.int64), direction=dirs)
    for i in range(N):
        o.add_photon(int(ids[i]), X[i], x[i], w[i], int(dirs[i]), 0, ts[i])
    g.step(120)
    o.step(120)
    cg, co = g.diag(spectrum=False)["counters"], o.counters()
    assert cg["pairs"] == co["pairs"] > 30
    a, b = P.leptons_gpu(g), P.leptons_oracle(o)
    assert np.array_equal(a["id"], b["id"])
    ga, gb = np.sqrt(1 + a["u"] ** 2), np.sqrt(1 + b["u"] ** 2)
    assert np.abs(ga / gb - 1.0).max() <= 5e-3
    assert np.median(np.abs(ga / gb - 1.0)) <= 1e-4
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("x0,b,n0", [(2.0 + 1e-9, 0.1, 0), (49.0, 1.0, -698)])
def test_pair_split_clamp_gives_finite_momenta(precision, x0, b, n0):
    """The clamp of a share below one rest mass (R27) acts on the energies:
    near the threshold x = 2, and at x = 49 where (1/49) 49 rounds below 1,
    400 conversions give finite momenta, clamped shares exactly at rest, the
    oracle's pair count, and energies summing to x."""
    cfg = dict(nx=512, boundary=O.BC_SURFACE, qed=1, qed_quantum=1, b=b, lambda_hat=1e-4, rho_hat=20.0,
               rate_mult=10.0, dx=0.1, dt=0.045, gap_length=51.2, ppc=1, density=1e-6)
    g, o = P.make_pair(cfg, precision, tile=64)
    N = 400
    ids = np.arange(1000, 1000 + N, dtype=np.uint64)
    X = 5.0 + 0.01 * np.arange(N)
    g.add_particles(2, ids, X, np.full(N, x0), np.full(N, 1e-3), np.zeros(N), n0=np.full(N, n0, np.int64),
                    direction=np.ones(N))
    for i in range(N):
        o.add_photon(int(ids[i]), X[i], x0, 1e-3, 1, n0, 0.0)
    g.step(1)
    o.step(1)
    assert g.diag(spectrum=False)["counters"]["pairs"] == o.counters()["pairs"] == N
    a = P.leptons_gpu(g)
    born = a["X"] > 2.0  # the pairs (the surface injects electrons into cell 0)
    u = a["u"][born]
    assert u.size == 2 * N and np.all(np.isfinite(u)) and np.all(u >= 0)
    assert np.count_nonzero(u == 0.0) > 0
    gam = np.sqrt(1 + u.astype(np.float64) ** 2)
    assert gam.sum() == pytest.approx(N * x0, rel=1e-9 if precision == "fp64" else 1e-5)
    g.close()
