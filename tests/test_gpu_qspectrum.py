"""The quantum photon spectrum option (qed_quantum) on the CUDA path: the
inverse against the oracle's exact inverse, one emission of each of 800
leptons at chi = 2 and a discharge against the oracle's from the same draws.

Tolerances: the FP64 state refines the table's estimate by Newton steps on
the exact survival (an exponential-integral reduction, qed_exact.cuh) and
the pair split on the exact distribution (tanh-sinh), so it follows the
oracle's exact inverses to rounding (1e-11 here, and the 1e-10 state parity
of a discharge).  The FP32 state reads the table: it interpolates ln s =
ln d / 3 over rows of ln chi (eight per decade, cubic) and the survival over
256 panels of s (cubic Hermite, panels crowded towards s = 0), an emulation
against the exact inverse below 2e-5 relative in xi for chi in [1e-6, 1e5],
plus float rounding of the survival (1e-7 absolute): relative 1e-3 for draws
U <= 0.999."""
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


@pytest.mark.parametrize("precision,rtol,umax", [("fp64", 1e-11, 1.0 - 1e-9), ("fp32", 1e-3, 0.999)])
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
    # near U = 1 both sides solve S(xi) = U S(0) where S(xi) and U S(0) differ
    # from S(0) by (1 - U) S(0) only: a relative error e of S moves xi by
    # e S(0)/(xi n(xi)), and with n ~ xi^(-2/3) at small xi that is
    # 3 e/(1 - U) relative; the sums for S carry e ~ 1e-14
    tol = np.maximum(rtol, 3e-14 / (1.0 - U)) if precision == "fp64" else rtol
    assert np.all(rel <= tol), (rel.max(), chi[rel.argmax()], U[rel.argmax()])
    g.close()


def test_qspectrum_inverse_needs_a_quantum_gap():
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300._abi import GapError
    g = Gap(P.gpu_params(dict(QCFG, qed_quantum=0)), precision="fp64", tile=16)
    with pytest.raises(GapError):
        g.qspectrum_inverse(torch.tensor([1.0]), torch.tensor([0.5]))
    g.close()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 2e-3)])
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
    """The electron's share of a conversion (gap_pair_split, the FP64
    evaluation): the table's estimate refined on the exact distribution
    equals the oracle's exact inverse to 1e-11 of the smaller share, far
    tail and Gaussian region (chi < 1e-3, where the estimate is the Gaussian
    limit) included."""
    g = _gap("fp64")
    cases = [(chi, U) for chi in (2e-4, 2e-3, 0.05, 1.0, 77.0, 1e3, 5e3)
             for U in (1e-6, 1e-5, 1e-4, 1e-3, 0.01, 0.2, 0.45, 0.5, 0.7, 0.999, 1 - 1e-5)]
    chi = np.array([c for c, _ in cases])
    U = np.array([u for _, u in cases])
    e = g.pair_split(torch.tensor(chi), torch.tensor(U)).cpu().numpy()
    ref = np.array([O.bw_split(c, u) for c, u in cases])
    small_gpu, small_ref = np.minimum(e, 1 - e), np.minimum(ref, 1 - ref)
    rel = np.abs(small_gpu / small_ref - 1.0)
    off = U != 0.5
    assert np.all((e[off] < 0.5) == (U[off] < 0.5))
    assert rel.max() <= 1e-11, (rel.max(), chi[rel.argmax()], U[rel.argmax()])
    g.close()


def test_quantum_pair_creation_matches_oracle():
    """Photons converting in a gap with qed_quantum (FP64 state): the same
    pairs at the same steps, the shares from the same draws on the exact
    distribution, and the pairs' states at 1e-10 of the oracle's."""
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
    P.compare_leptons(a, b, 1e-10, "pairs of the quantum split")
    g.close()


def test_config1_quantum_parity_first_200_steps():
    """Config 1 with the quantum photon spectrum and pair split (FP64): E and
    every lepton within 1e-10 of the oracle with identical event counters over
    the first 200 steps (the state parity criterion), the emissions drawn
    on the exact spectrum."""
    cfg = dict(P.CONFIG1, qed_quantum=1)
    g, o = P.make_pair(cfg, "fp64", tile=64)
    for n in (100, 200):
        g.step(n - o.stepno)
        o.step(n - o.stepno)
        P.compare_counters(g.diag(spectrum=False)["counters"], o.counters(), f"step {n}")
        P.compare_field(g.field(), o.E(), 1e-10, f"E step {n}")
        P.compare_leptons(P.leptons_gpu(g), P.leptons_oracle(o), 1e-10, f"leptons step {n}")
    assert o.counters()["emit_events"] > 300
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
