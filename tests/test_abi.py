"""The C-ABI library loads and exports every entry point include/gap.h
declares; host-side layout and validation work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|int64_t|size_t|const char \*)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2608_21920_b300 import _abi
    L = _abi.lib()
    declared = _declared()
    assert len(declared) >= 15
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(_abi.EXPORTED) == declared


def test_workspace_bytes_and_validation_without_gpu():
    from paper_2608_21920_b300 import _abi as A
    from paper_2608_21920_b300.gap import make_params
    L = A.lib()
    p = make_params(nx=512, ppc=16, init=A.GAP_INIT_COLD, qed=1, cap=200000)
    cfg = A.GapConfig(precision=A.GAP_FP32_STATE, tile=64)
    n = C.c_size_t(0)
    assert L.gap_workspace_bytes(C.byref(p), 1, C.byref(cfg), C.byref(n)) == A.GAP_OK
    assert 1e6 < n.value < 1e9
    bad = make_params(nx=512, dx=0.1, dt=0.06)  # c dt/dx >= 1/2
    assert L.gap_workspace_bytes(C.byref(bad), 1, C.byref(cfg), C.byref(n)) == A.GAP_EINVAL
    big = make_params(nx=1 << 20, ppc=400, init=A.GAP_INIT_PAIR_THERMAL, boundary=A.GAP_BC_PERIODIC,
                      theta=0.1, density=1.0)
    cfg2 = A.GapConfig(precision=A.GAP_FP32_STATE, tile=256)
    assert L.gap_workspace_bytes(C.byref(big), 1, C.byref(cfg2), C.byref(n)) == A.GAP_OK
    assert n.value < 100e9  # fits the 270 GB of HBM with room to spare
    assert L.gap_status_string(A.GAP_ECAP).decode() == "particle storage exhausted"


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2608_21920_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("CPU oracle", ""), f
