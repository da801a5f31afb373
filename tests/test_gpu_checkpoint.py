"""Checkpoint and resume through the C ABI (gap_save / gap_load): a state
saved mid-discharge and loaded into a fresh handle (another workspace) steps
on exactly as the original handle does; a state of another layout is
refused and leaves the handle usable."""
import numpy as np
import pytest

from tests import _pair as P

pytestmark = pytest.mark.gpu


def _snapshot(g):
    d = g.diag(spectrum=False)
    c = {k: d["counters"][k] for k in P.COUNTER_KEYS}
    lep = P.leptons_gpu(g)
    ph = g.particles(2)
    o = np.argsort(ph["id"])
    return dict(E=g.field(), counters=c, step=d["step"], lep=lep, ph={k: v[o] for k, v in ph.items()})


def test_resume_continues_exactly():
    from paper_2608_21920_b300 import Gap, _abi as A
    params = P.gpu_params(P.SMALL_DISCHARGE)
    a = Gap(params, precision="fp32", tile=32)
    a.step(560)  # pairs have started
    state = a.save()
    a.step(200)
    ref = _snapshot(a)
    assert ref["counters"]["pairs"] > 0 and ref["counters"]["photons"] > 0
    a.close()

    b = Gap(params, precision="fp32", tile=32)
    b.load(state)
    assert b.steps_done == 560
    b.step(200)
    got = _snapshot(b)
    b.close()
    # FP32 state: exact integer charge, draws keyed by id and step: bitwise equal
    assert got["step"] == ref["step"] and got["counters"] == ref["counters"]
    assert np.array_equal(got["E"], ref["E"])
    for k in ("id", "X", "u", "w", "tau", "q"):
        assert np.array_equal(got["lep"][k], ref["lep"][k]), k
    for k in ("id", "X", "x", "w", "tau_acc", "tau_star"):
        assert np.array_equal(got["ph"][k], ref["ph"][k]), k


def test_state_of_another_layout_is_refused():
    from paper_2608_21920_b300 import Gap, _abi as A
    a = Gap(P.gpu_params(P.SMALL_DISCHARGE), precision="fp32", tile=32)
    a.step(5)
    state = a.save()
    a.close()
    c = Gap(P.gpu_params(P.SMALL_DISCHARGE), precision="fp32", tile=16)  # other tiles
    with pytest.raises(A.GapError):
        c.load(state if state.size == A.lib().gap_state_bytes(c.handle) else state[:0])
    c.step(5)  # nothing was copied: the handle runs on
    assert c.diag(spectrum=False)["gauss_residual"] < 1e-10
    c.close()
