"""Failures reported, not faulted: a particle store that fills up makes the
library flag the condition on the device (bounds-checked appends), and the
next call that reads the control block returns GAP_ECAP with the reason; the
handle keeps that status, and the GPU stays usable for other handles."""
import pytest

from tests import _pair as P

pytestmark = pytest.mark.gpu


def _usable_afterwards():
    from paper_2608_21920_b300 import Gap
    h = Gap(P.gpu_params(dict(P.SMALL_DISCHARGE, qed=0)), precision="fp64", tile=32)
    h.step(10)
    assert h.diag(spectrum=False)["gauss_residual"] < 1e-10
    h.close()


def test_photon_store_exhaustion_is_reported():
    from paper_2608_21920_b300 import Gap, _abi as A
    g = Gap(P.gpu_params(P.SMALL_DISCHARGE), precision="fp64", tile=32, photon_capacity=8)
    with pytest.raises(A.GapError, match="photon storage exhausted"):
        for _ in range(24):
            g.step(50)
            g.diag(spectrum=False)
    with pytest.raises(A.GapError, match="exhausted"):  # the status stays on the handle
        g.field()
    g.close()
    _usable_afterwards()


def test_lepton_store_exhaustion_is_reported():
    from paper_2608_21920_b300 import Gap, _abi as A
    # the store holds the initial layout only; the discharge's pairs overflow it
    g = Gap(P.gpu_params(P.SMALL_DISCHARGE), precision="fp64", tile=32, lepton_capacity=1, rebin_every=16)
    with pytest.raises(A.GapError, match="exhausted"):
        for _ in range(40):
            g.step(50)
            g.diag(spectrum=False)
    g.close()
    _usable_afterwards()


def test_bulk_copy_wait_runs_out_into_an_error():
    """The bulk-copy push (variant 4) waits on each copy stage with a bounded
    poll loop; the test hook leaves a stage unissued so that the wait runs out
    (after a short limit): the kernel records it and returns, the next call
    reports GAP_ETIMEOUT, and the GPU stays usable."""
    import oracle as O
    from paper_2608_21920_b300 import Gap, _abi as A
    cfg = dict(nx=2048, ppc=16, dx=0.1, dt=0.045, theta=0.1, density=1.0, init=O.INIT_PAIR_THERMAL,
               boundary=O.BC_PERIODIC, seed=0)
    g = Gap(P.gpu_params(cfg), precision="fp32", tile=256, threads=256, variant=4)
    g.step(2)
    assert g.diag(spectrum=False)["gauss_residual"] < 1e-10  # the variant runs normally first
    A.check(A.lib().gap_hold_copies(g.handle, 1), g.handle, "gap_hold_copies")
    g.step(1)
    with pytest.raises(A.GapError, match="never completed"):
        g.diag(spectrum=False)
    g.close()
    _usable_afterwards()
