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


def test_option_checks_and_em_layout_without_gpu():
    """Host-side validation of the transverse-field and proton options, and
    the five FP64 node arrays (E_y, E_z, B_y, B_z, dt jv_h) the fields add."""
    from paper_2608_21920_b300 import _abi as A
    from paper_2608_21920_b300.gap import make_params
    L = A.lib()
    n = C.c_size_t(0)
    f64 = A.GapConfig(precision=A.GAP_FP64_PLAIN, tile=64)
    f32 = A.GapConfig(precision=A.GAP_FP32_STATE, tile=64)

    def code(cfg=f64, **kw):
        p = make_params(**dict(dict(nx=512, ppc=4, init=A.GAP_INIT_COLD), **kw))
        return L.gap_workspace_bytes(C.byref(p), 1, C.byref(cfg), C.byref(n))

    good = [dict(em=1), dict(em=1, beta_y=3e-6), dict(em=1, beta_y=0.6, beta_z=0.7), dict(em=1, pml_cells=16),
            dict(em=1, pml_cells=256, pml_sigma=5.0), dict(protons=1), dict(protons=1, init=A.GAP_INIT_GAP_PROTONS),
            dict(protons=1, cap=1000)]
    bad = [dict(beta_y=1e-3), dict(pml_cells=4), dict(em=1, beta_y=0.8, beta_z=0.6), dict(em=1, beta_z=float("inf")),
           dict(em=1, pml_cells=257), dict(em=1, pml_cells=-1), dict(em=3), dict(em=1, pml_cells=8, pml_sigma=-2.0),
           dict(em=1, pml_cells=8, boundary=A.GAP_BC_PERIODIC, init=A.GAP_INIT_EMPTY, ppc=0),
           dict(protons=2), dict(init=A.GAP_INIT_GAP_PROTONS),
           dict(protons=1, init=A.GAP_INIT_GAP_PROTONS, boundary=A.GAP_BC_PERIODIC), dict(protons=1, m_ion=-1.0)]
    for kw in good:
        assert code(**kw) == A.GAP_OK, kw
    for kw in bad:
        assert code(**kw) == A.GAP_EINVAL, kw
    assert code(f32, em=1, beta_y=0.1) == A.GAP_OK
    assert code(f32, protons=1) == A.GAP_OK
    assert code(nx=512) == A.GAP_OK
    plain = n.value
    assert code(nx=512, em=1) == A.GAP_OK
    assert n.value - plain >= 5 * 8 * 513


def test_struct_layouts_match_the_header(tmp_path):
    """gap.h compiles as strict C99, and the binding's ctypes structures have
    the header's size and field offsets (a field out of order on either side
    would shift every later field)."""
    import shutil
    import subprocess
    from paper_2608_21920_b300 import _abi as A
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    STRUCTS = (("gap_params", A.GapParams), ("gap_config", A.GapConfig), ("gap_counters", A.GapCounters),
               ("gap_diag_out", A.GapDiagOut))
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gap.h"', "int main(void) {"]
    for ctype, st in STRUCTS:
        lines.append(f'  printf("{ctype} size %zu\\n", sizeof({ctype}));')
        for name, _ in st._fields_:
            lines.append(f'  printf("{ctype} {name} %zu\\n", offsetof({ctype}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(t, n): int(v) for t, n, v in (l.split() for l in out if l)}
    for ctype, st in STRUCTS:
        assert got[(ctype, "size")] == C.sizeof(st), ctype
        for name, _ in st._fields_:
            assert got[(ctype, name)] == getattr(st, name).offset, (ctype, name)
