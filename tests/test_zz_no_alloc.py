"""The allocation-free spectrum entry point against the regular diagnostic.

gap_power_spectrum_noalloc serves callers that cannot allocate device
memory: it works from the caller's input and output buffers and a fixed
array inside the library.  Called through the C ABI twice in a row, it must
give the spectrum that gap_diag computes with its own workspace.  This file
is collected last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_spectrum_matches_diag_twice():
    import torch

    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300 import _abi as A
    from tests import _pair as P

    g = Gap(P.gpu_params(P.SMALL_DISCHARGE), precision="fp64", tile=32)
    g.step(300)
    ref = g.diag(spectrum=True)["spectrum"]
    p = g.param_dicts[0]
    ng = min(int(math.floor(p["gap_length"] / p["dx"])) + 1, g.nnode())
    E = torch.tensor(g.field()[:ng], dtype=torch.float64, device="cuda")
    out = torch.empty(ref.size, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = A.lib()
    for _ in range(2):
        out.fill_(float("nan"))
        st = L.gap_power_spectrum_noalloc(C.c_void_p(E.data_ptr()), ng, C.c_void_p(out.data_ptr()), stream)
        assert st == A.GAP_OK
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-14 * ref.max())
    big = torch.zeros(40000, dtype=torch.float64, device="cuda")
    sink = torch.empty(32769 * 2, dtype=torch.float64, device="cuda")
    assert L.gap_power_spectrum_noalloc(C.c_void_p(big.data_ptr()), 40000, C.c_void_p(sink.data_ptr()),
                                        stream) == A.GAP_ETOOBIG
