"""The C-ABI library loads and exports every symbol include/fftg.h declares.

No compute calls: this runs without a GPU.
"""
import os
import re

import pytest

from paper_1601_05970_gb300 import build, fftg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fftg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fftg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fftg.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in fftg.SIGNATURES, n


def test_host_only_entry_points(lib):
    import ctypes as C
    assert lib.fftg_version().startswith(b"fftg")
    o = fftg.default_options()
    assert o.precision == fftg.FFTG_MIXED and o.max_cg == 2000 and o.nrhs_tangent == 6
    b = C.c_size_t()
    assert lib.fftg_workspace_size(15, C.byref(o), C.byref(b)) == 0 and b.value > 0
    # even N, N not 3^a 5^b, N too large: rejected before any device work
    for bad in (0, 2, 14, 7, 21, 729):
        assert lib.fftg_workspace_size(bad, C.byref(o), C.byref(b)) == fftg.FFTG_EINVAL
    h = C.c_void_p()
    assert lib.fftg_create(C.byref(h), 14, None, 1, None, None) == fftg.FFTG_EINVAL


def test_workspace_grows_with_precision_and_rhs(lib):
    o = fftg.default_options()
    mixed = fftg.workspace_size(45, o)
    o.precision = fftg.FFTG_FP64
    f64 = fftg.workspace_size(45, o)
    o.nrhs_tangent = 0
    f64_norhs = fftg.workspace_size(45, o)
    assert f64 > mixed > 0 and f64 > f64_norhs
