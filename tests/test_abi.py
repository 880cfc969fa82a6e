"""The C-ABI library loads and exports every function include/vest.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vest.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vest_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_02603_gb300 import build as B
    from paper_1904_02603_gb300 import vest as V
    B.build()
    return V.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["vest_build_index", "vest_sweep_factors", "vest_sweep_core", "vest_responsibility",
                     "vest_prune", "vest_loss", "vest_autosearch"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1904_02603_gb300 import vest as V
    assert set(V.exported_symbols()) == set(declared_functions())


def test_version_and_host_side_validation(lib):
    import ctypes as C
    from paper_1904_02603_gb300 import vest as V
    assert b"sm_103a" in lib.vest_version()
    # host-side argument checks run without touching the GPU
    t = V.vest_tensor()
    t.order = 1
    assert lib.vest_index_workspace_bytes(C.byref(t)) == 0
    h = C.c_void_p()
    assert lib.vest_build_index(None, None, 0, C.byref(h), None) == 1
    assert lib.vest_build_index(C.byref(t), None, 0, C.byref(h), None) == 1
    assert b"order" in lib.vest_last_error()
    m = V.vest_model()
    m.order = 3
    assert lib.vest_normalize(C.byref(m), None, 0, None) == 1


def test_struct_layouts_match_header():
    import ctypes as C
    from paper_1904_02603_gb300 import vest as V
    # offsets fixed by the C declarations in include/vest.h (LP64)
    assert V.vest_tensor.dims.offset == 8 and V.vest_tensor.idx.offset == 96
    assert V.vest_model.ranks.offset == 88 and V.vest_model.factor.offset == 128
    assert V.vest_model.core.offset == 288 and C.sizeof(V.vest_model) == 304
    assert V.vest_params.lambda_.offset == 8 and V.vest_report.re_hist.offset == 8


def test_every_struct_field_matches_the_c_layout(tmp_path):
    """Offsets and sizes of every field of every struct the binding mirrors, as gcc lays them out
    from include/vest.h, equal the ctypes declarations."""
    import ctypes as C
    import shutil
    import subprocess
    from paper_1904_02603_gb300 import vest as V
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    structs = [V.vest_tensor, V.vest_model, V.vest_mode_view, V.vest_params, V.vest_report]
    lines = ['#include <stdio.h>', '#include "vest.h"', "int main(void) {"]
    for st in structs:
        for name, _ in st._fields_:
            cname = "lambda" if name == "lambda_" else name
            lines.append(f'  printf("{st.__name__} {name} %zu %zu\\n", offsetof({st.__name__}, {cname}), '
                         f"sizeof((({st.__name__}*)0)->{cname}));")
        lines.append(f'  printf("{st.__name__} SIZE %zu 0\\n", sizeof({st.__name__}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    by_struct = {st.__name__: st for st in structs}
    out = [line for line in out if line]
    assert len(out) == sum(len(st._fields_) + 1 for st in structs)
    for line in out:
        sname, field, off, size = line.split()
        st = by_struct[sname]
        if field == "SIZE":
            assert C.sizeof(st) == int(off), sname
            continue
        f = getattr(st, field)
        assert (f.offset, f.size) == (int(off), int(size)), (sname, field, f.offset, f.size, off, size)
