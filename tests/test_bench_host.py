"""bench.py's host logic without a GPU: the workload options reach the gap
parameters, and every option combination passes the library's own
validation (gap_workspace_bytes runs on the host)."""
import ctypes as C
import importlib

import pytest


@pytest.fixture
def bench():
    import bench as b
    b = importlib.reload(b)  # module-level workload state starts fresh
    yield b
    importlib.reload(b)


@pytest.mark.parametrize("opts", [(0, 0.0, 0, 0), (8, 0.3, 1, 0), (0, 0.0, 0, 1), (8, 0.3, 1, 1)])
def test_options_reach_the_parameters_and_validate(bench, opts):
    from paper_2608_21920_b300 import _abi as A
    from paper_2608_21920_b300.gap import make_params
    filter_passes, theta, quantum, em = opts
    bench.set_setup(filter_passes, theta, quantum, em)
    params = bench.batch_params(8)
    assert all(p["filter_passes"] == filter_passes and p["inject_theta"] == theta for p in params)
    assert all(p["qed_quantum"] == quantum and p["em"] == em for p in params)
    if em:
        assert all(p["beta_y"] == bench.BETA_ROT for p in params)
        assert all(p.get("pml_cells", 0) == (bench.PML_CELLS if p["boundary"] == A.GAP_BC_SURFACE else 0)
                   for p in params)
        assert bench.WORKLOAD["em"] == 1 and "co-rotating" in bench.WORKLOAD_NAME
    arr = (A.GapParams * len(params))(*[make_params(**p) for p in params])
    n = C.c_size_t(0)
    for prec in (A.GAP_FP32_STATE, A.GAP_FP64_PLAIN):
        cfg = A.GapConfig(precision=prec, tile=128)
        assert A.lib().gap_workspace_bytes(arr, len(params), C.byref(cfg), C.byref(n)) == A.GAP_OK
    one = make_params(**bench.WORKLOAD)
    cfg = A.GapConfig(precision=A.GAP_FP32_STATE, tile=256)
    assert A.lib().gap_workspace_bytes(C.byref(one), 1, C.byref(cfg), C.byref(n)) == A.GAP_OK
