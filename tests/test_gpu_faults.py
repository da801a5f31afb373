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
