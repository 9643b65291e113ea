"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/fem.h declares
(no GPU needed: no compute call is made)."""
import os
import re

import pytest

from paper_2409_20380_gb300 import build, fem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:fem_status|void|const char\s*\*)\s*\**\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libfem():
    build.build()
    return fem.lib()


def test_header_and_binding_agree():
    assert sorted(fem.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(libfem):
    for name in _declared():
        assert hasattr(libfem, name), name


def test_defaults_and_errors_without_gpu(libfem):
    o = fem.fem_opts_default()
    assert o.tol == 1e-8 and o.precision == fem.FEM_FP64 and o.s_max == 32
    # the last fields read back their documented defaults (the binding's struct layout matches the header's)
    assert o.wait_budget == 1048576 and o.cpu_predictor == 0 and o.inner_margin == 0.5
    assert o.inner_product == fem.FEM_INNER_FP32 and o.pred_guard == 1
    # argument errors are reported without touching a device
    st = libfem.fem_mesh_destroy(None)
    assert st == fem.FEM_ERR_ARG
    assert "null" in fem.fem_last_error()
