"""The C ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(labfm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    import __graft_entry__ as g
    return g._builder().build()


def test_library_exports_every_declared_symbol(built_lib):
    declared = _declared_functions()
    assert "labfm_build_stencils" in declared and "labfm_rk_step" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(labfm_\w+)\b", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_binding_loads_and_covers_the_header(built_lib):
    import paper_2102_02019_gb300 as lb
    assert lb.lib.labfm_abi_version() == 2
    assert lb.lib.labfm_last_error() == b""
    declared = set(_declared_functions())
    assert declared <= set(lb.exported_symbols()), declared - set(lb.exported_symbols())


def test_errors_are_reported_without_a_gpu(built_lib):
    import ctypes
    import paper_2102_02019_gb300 as lb
    # argument validation happens on the host before any CUDA call
    nnz = ctypes.c_int64(0)
    rc = lb.lib.labfm_build_stencils(None, None, 10, 1.0, 1.0, 3, None, None, 0, ctypes.byref(nnz), None)
    assert rc == 1 and b"null" in lb.lib.labfm_last_error()
    rc = lb.lib.labfm_build_weights(1, 1, 1, 10, 1.0, 1.0, 3, 1, 1, 10, 5, 1, 1, None, 1, None, None)
    assert rc == 1 and b"order m" in lb.lib.labfm_last_error()
    rc = lb.lib.labfm_rhs(None, 1, 2, None, None)
    assert rc == 1
