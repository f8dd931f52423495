"""The C-ABI library loads and exports every symbol include/*.h declares.

No compute calls: this runs without a GPU.
"""
import os
import re

import numpy as np
import pytest

from paper_1601_05970_gb300 import build, fftg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
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


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of the header's structs: size and every field offset,
    # as a C compiler lays them out (host gcc; no GPU)
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fftg_phase": fftg.fftg_phase, "fftg_options": fftg.fftg_options,
               "fftg_stats": fftg.fftg_stats, "fftg_result": fftg.fftg_result,
               "fftg_svk_phase": fftg.fftg_svk_phase}
    cname = {"lambda_": "lambda"}   # a Python keyword in the ctypes mirror
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fftg_fs.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {cname.get(f[0], f[0])}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


def test_noalloc_rejects_rate_dependent_phases(lib):
    # checked on the host before any device work
    import ctypes as C
    from paper_1601_05970_gb300 import inputs as I
    mats = fftg.phase_array((I.ViscoPlastic(0.833, 0.386, 0.0386, 0.1, 0.1, 0.3),))
    E = np.zeros(6)
    mean = np.zeros(6)
    dummy = C.c_void_p(1)   # never dereferenced
    d6 = E.ctypes.data_as(C.POINTER(C.c_double))
    m6 = mean.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.fftg_constitutive_noalloc(15, d6, dummy, dummy, dummy, dummy, 1, mats,
                                         fftg.FFTG_FP64, None, dummy, None, None, m6,
                                         None) == fftg.FFTG_EINVAL


def test_create_rejects_invalid_phases(lib):
    # model-specific parameter checks happen before any device work
    import ctypes as C
    from paper_1601_05970_gb300 import inputs as I
    ph = np.zeros(27, np.uint8)
    bad = [I.Phase(0.833, 0.386, 0.003, 0.01, 0.0),            # n = 0
           I.Phase(0.833, 0.0, 0.003, 0.01),                    # G = 0
           I.NonlinearElastic(0.833, 0.2, 0.0, 10.0),           # eps0 = 0
           I.ViscoPlastic(0.833, 0.386, 0.0386, 0.1, 0.0, 0.3)]  # t0 = 0
    for m in bad:
        h = C.c_void_p()
        assert lib.fftg_create(C.byref(h), 3, ph.ctypes.data_as(C.POINTER(C.c_uint8)), 1,
                               fftg.phase_array((m,)), None) == fftg.FFTG_EINVAL, m
    o = fftg.default_options()
    assert o.dt == 1.0
    o.dt = 0.0
    h = C.c_void_p()
    assert lib.fftg_create(C.byref(h), 3, ph.ctypes.data_as(C.POINTER(C.c_uint8)), 1,
                           fftg.phase_array((I.SOFT,)), C.byref(o)) == fftg.FFTG_EINVAL


def test_finite_strain_create_rejects_bad_arguments(lib):
    # host-side checks, before any device work
    import ctypes as C
    ph = np.zeros(27, np.uint8)
    php = ph.ctypes.data_as(C.POINTER(C.c_uint8))
    good = fftg.svk_array(((0.5, 0.4),))
    h = C.c_void_p()
    for m in (((-0.1, 0.4),), ((0.5, 0.0),), ((float("nan"), 0.4),)):
        assert lib.fftg_fs_create(C.byref(h), 3, php, 1, fftg.svk_array(m), None) == fftg.FFTG_EINVAL
    for bad_n in (2, 7, 729):
        assert lib.fftg_fs_create(C.byref(h), bad_n, php, 1, good, None) == fftg.FFTG_EINVAL
    ph2 = ph.copy()
    ph2[5] = 1                                                   # phase id >= nphase
    assert lib.fftg_fs_create(C.byref(h), 3, ph2.ctypes.data_as(C.POINTER(C.c_uint8)), 1, good,
                              None) == fftg.FFTG_EINVAL
    o = fftg.default_options()
    o.solver = fftg.FFTG_SOLVER_RICHARDSON                       # CG only
    assert lib.fftg_fs_create(C.byref(h), 3, php, 1, good, C.byref(o)) == fftg.FFTG_EINVAL
    o = fftg.default_options()
    o.workspace = C.c_void_p(256)                                # own memory only
    assert lib.fftg_fs_create(C.byref(h), 3, php, 1, good, C.byref(o)) == fftg.FFTG_EINVAL
    b = C.c_size_t()
    o = fftg.default_options()
    assert lib.fftg_fs_workspace_size(45, C.byref(o), C.byref(b)) == 0
    mixed = b.value
    o.precision = fftg.FFTG_FP64
    assert lib.fftg_fs_workspace_size(45, C.byref(o), C.byref(b)) == 0
    assert b.value > mixed > 0
    assert lib.fftg_fs_profile_kinds() > 0 and lib.fftg_fs_profile_name(0).startswith(b"fs_")
