"""The asynchronous field readback (gap_get_field_async): E copied to pinned
host memory on a second stream, while the next steps run, equals what the
synchronous readback returns at the same step of a twin run (bit for bit
with the FP32 state, whose deposit is an exact integer sum; to rounding
with FP64, whose atomic sums depend on their order), so the steps that
follow a readback do not change the copy it made."""
import numpy as np
import pytest
import torch

import oracle as O
from tests import _pair as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_async_readback_matches_the_synchronous_one(precision):
    from paper_2608_21920_b300 import Gap
    cfg = dict(P.CONFIG1, cap=200000)
    a = Gap(P.gpu_params(cfg), precision=precision, tile=64)
    b = Gap(P.gpu_params(cfg), precision=precision, tile=64)
    nn = a.nnode()
    copy = torch.cuda.Stream()
    outs = [torch.empty(nn, dtype=torch.float64, pin_memory=True) for _ in range(12)]
    ref = []
    for k in range(12):
        a.step(25)
        a.field_async(outs[k], copy)
        b.step(25)
        ref.append(b.field())
    copy.synchronize()
    torch.cuda.synchronize()
    for k in range(12):
        if precision == "fp32":
            assert np.array_equal(outs[k].numpy(), ref[k]), k
        else:
            P.compare_field(outs[k].numpy(), ref[k], 1e-10, f"copy {k}")
    if precision == "fp32":
        assert np.array_equal(a.field(), b.field())
    assert not np.array_equal(ref[0], ref[-1])  # E moved between the copies
    a.close()
    b.close()


def test_async_readback_checks_its_arguments():
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300 import _abi as A
    import ctypes as C
    g = Gap(P.gpu_params(dict(nx=64, dx=0.1, dt=0.045, boundary=O.BC_SURFACE)), precision="fp64", tile=16)
    out = torch.empty(g.nnode(), dtype=torch.float64, pin_memory=True)
    copy = torch.cuda.Stream()
    L = A.lib()
    ptr = C.c_void_p(out.data_ptr())
    assert L.gap_get_field_async(g.handle, 1, ptr, out.numel(), g.stream(), C.c_void_p(copy.cuda_stream)) == A.GAP_EINVAL
    assert L.gap_get_field_async(g.handle, 0, ptr, out.numel() - 1, g.stream(), C.c_void_p(copy.cuda_stream)) == A.GAP_EINVAL
    g.close()
