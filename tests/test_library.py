"""The C-ABI library builds, loads and exports every entry point that
include/gdr.h declares (no compute: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_0707_0502_gb300 import build
    build.build()
    import paper_0707_0502_gb300 as g
    return g


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gdr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gdr_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for need in ("gdr_create", "gdr_op_wilson", "gdr_op_csr", "gdr_solve_multishift", "gdr_solve_proj",
                 "gdr_arnoldi_step", "gdr_dense_gmres_sh", "gdr_dense_restart", "gdr_basis_update"):
        assert need in names


def test_every_declared_symbol_is_exported(built):
    L = ctypes.CDLL(built.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps every declared entry point
    assert set(declared_functions()) <= set(built._SIGS)


def test_params_default_and_status_strings(built):
    p = built.gdr_params_default()
    assert (p.m, p.k, p.tol, p.prec) == (40, 20, 1e-8, built.GDR_PREC_FP64)
    L = built.lib()
    assert L.gdr_status_string(built.GDR_ENOCONV) == b"GDR_ENOCONV"


def test_create_without_gpu_fails_loudly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = built.lib().gdr_create(ctypes.byref(h), 0, None)
    assert st == built.GDR_ECUDA
    assert h.value is None
    assert built.lib().gdr_last_error(None)


def test_struct_layouts_match_header(built, tmp_path):
    """Offsets of every field of the ABI structs, from the C compiler vs ctypes."""
    fields = {"gdr_params": [f for f, _ in built.gdr_params._fields_],
              "gdr_report": [f for f, _ in built.gdr_report._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gdr.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, cls in (("gdr_params", built.gdr_params), ("gdr_report", built.gdr_report)):
        assert int(out[st]) == ctypes.sizeof(cls)
        for f in fields[st]:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
