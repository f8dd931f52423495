"""fftg_constitutive_noalloc, the entry point for callers that cannot
allocate device memory, against the handle-based fftg_op_constitutive.

Such a caller (a host code whose own pool already holds the device memory)
passes every buffer itself; the call's only scratch is a fixed array inside
the library. Both calls run the same stress update, so the stress fields
must agree to the 1e-14 relative tolerance of the constitutive parity test,
and the returned mean stress must be the mean of that field. Two calls in a
row check that the shared scratch left by the first call does not leak into
the second.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1601_05970_gb300 import build
    build.build()
    return fftg.load()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_constitutive_matches_handle_call_twice(lib):
    N = 15
    V = N ** 3
    ph, _, _ = I.random_spheres(N, 0.3, 11, r_min=2.0, r_max=4.0)
    cell = fftg.Cell(N, ph, I.TWO_PHASE, precision="fp64", nrhs_tangent=0)
    for dE in I.shear_path(0.02, 20)[:3]:           # build up a plastic history
        cell.step(dE, 1e-5, 1e-8)
    state = cell.get_state()
    E = state[:6].copy()
    dev = dict(dtype=torch.float64, device="cuda")
    eps = torch.tensor(state[6:6 + 6 * V], **dev)
    eps_p = torch.tensor(state[6 + 6 * V:6 + 12 * V], **dev)
    epbar = torch.tensor(state[6 + 12 * V:6 + 13 * V], **dev)
    assert float(epbar.max()) > 0.0
    phase = torch.tensor(ph.reshape(-1), dtype=torch.uint8, device="cuda")
    mats = (fftg.fftg_phase * 2)(*[fftg.fftg_phase(*m.as_tuple()) for m in I.TWO_PHASE])
    stream = torch.cuda.current_stream().cuda_stream
    for dE in (np.array([0, 0, 0, 0, 0, 0.0015]), np.array([0.001, -0.0004, 0.0002, 0.0003, 0.0, 0.0008])):
        ref = cell.constitutive(dE=dE).cpu().numpy()
        sig = torch.full((6 * V,), np.nan, **dev)
        mean = np.zeros(6)
        Et = E + dE
        rc = lib.fftg_constitutive_noalloc(
            N, Et.ctypes.data_as(C.POINTER(C.c_double)), _ptr(eps), _ptr(eps_p), _ptr(epbar),
            _ptr(phase), 2, mats, fftg.FFTG_FP64, None, _ptr(sig), None, None,
            mean.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream))
        assert rc == fftg.FFTG_OK
        got = sig.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
        ref_mean = ref.reshape(6, V).mean(axis=1)
        assert np.abs(mean - ref_mean).max() <= 1e-14 * np.abs(ref_mean).max()
    cell.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    mats = (fftg.fftg_phase * 1)(fftg.fftg_phase(1.0, 0.5, 0.01, 0.0, 1.0))
    E = np.zeros(6)
    mean = np.zeros(6)
    dummy = C.c_void_p(1)  # never dereferenced: the size check comes first
    d6 = E.ctypes.data_as(C.POINTER(C.c_double))
    m6 = mean.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.fftg_constitutive_noalloc(245, d6, dummy, dummy, dummy, dummy, 1, mats,
                                         fftg.FFTG_FP64, None, dummy, None, None, m6,
                                         None) == fftg.FFTG_EINVAL
    assert lib.fftg_constitutive_noalloc(15, d6, dummy, dummy, dummy, dummy, 257, mats,
                                         fftg.FFTG_FP64, None, dummy, None, None, m6,
                                         None) == fftg.FFTG_EINVAL
