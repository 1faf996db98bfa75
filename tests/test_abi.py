"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; calls fail cleanly (status codes, no crash) when no
GPU is present or arguments are invalid."""
import ctypes
import glob
import os
import re

import pytest

import paper_2301_04642_gb300 as fe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names.update(re.findall(r"FE_API\s+[\w\s\*]+?\b(fe_\w+)\s*\(", txt))
    return sorted(names)


def test_headers_declare_the_abi():
    names = declared_symbols()
    for want in ("fe_create", "fe_destroy", "fe_solve", "fe_solve_batch", "fe_submit", "fe_poll",
                 "fe_last_error_string", "fe_k_gershgorin", "fe_k_sym_square"):
        assert want in names


def test_library_exports_every_declared_symbol():
    L = fe.load()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_null_context_calls_fail_cleanly():
    L = fe.load()
    r = fe.FeResult()
    p = fe.FeProblem()
    assert L.fe_solve(None, ctypes.byref(p), ctypes.byref(r)) == fe.FE_EINVAL
    assert L.fe_solve_batch(None, 0, None, None) == fe.FE_EINVAL
    assert L.fe_destroy(None) == fe.FE_OK
    assert L.fe_create(None, None) == fe.FE_EINVAL
    assert b"NULL" in L.fe_last_error_string(None)


def test_create_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fe.FeError) as ei:
        fe.Context()
    assert ei.value.status == fe.FE_ECUDA


def test_struct_layouts_match_header(tmp_path):
    # compile the public header with the host C compiler and compare every
    # field offset with the binding's ctypes mirror
    import subprocess
    fields = {"fe_problem": fe.FeProblem, "fe_result": fe.FeResult, "fe_config": fe.FeConfig}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fe.h"', "int main(void){"]
    for cname, cls in fields.items():
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f, _ in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = []
    for cname, cls in fields.items():
        want.append(ctypes.sizeof(cls))
        want.extend(getattr(cls, f).offset for f, _ in cls._fields_)
    assert got == want
