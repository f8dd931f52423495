"""fftg_constitutive_noalloc, the entry point for callers that cannot
allocate device memory, against the FP64 oracle and against the
handle-based fftg_op_constitutive.

Such a caller (a host code whose own pool already holds the device memory)
passes every buffer itself; the call's only scratch is a fixed array inside
the library. Checked on two calls in a row, so that the shared scratch left
by the first call does not leak into the second:
* the stress field against the oracle's J2 update and against the handle
  call, to the 1e-14 relative tolerance of the constitutive parity test, and
  the returned mean stress against the mean of that field;
* the updated history (plastic strain and accumulated plastic strain)
  against the oracle, to 1e-14 of its largest value;
* the compact tangent written in FP64 and in FP32: C : p rebuilt from it for
  a random p against the oracle's consistent tangent, to 1e-13 (FP64) and
  to FP32 rounding, 1e-6 (FP32), of |C| |p|.
A phase id at or above nphase is reported as FFTG_EINVAL.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import fftg_oracle as O
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
    return C.c_void_p(0 if t is None else t.data_ptr())


def _apply_compact(t7, p):
    """C : p from the documented compact tangent [7][V] (K', 2G_eff, w11,
    w22, w23, w13, w12; C = |K'| I(x)I + 2G_eff I_d - sign(K') w(x)w,
    w33 = -(w11 + w22), Frobenius product with shears counted twice)."""
    K, g2, w11, w22, w23, w13, w12 = t7
    w = np.stack([w11, w22, -(w11 + w22), w23, w13, w12])
    tr = p[0] + p[1] + p[2]
    wp = w[0] * p[0] + w[1] * p[1] + w[2] * p[2] + 2.0 * (w[3] * p[3] + w[4] * p[4] + w[5] * p[5])
    sgn = np.where(K < 0, -1.0, 1.0)
    s = g2 * p
    s[:3] += (np.abs(K) * tr - g2 * tr / 3.0)[None]
    return s - sgn * wp * w


def test_noalloc_constitutive_matches_oracle_and_handle_call_twice(lib):
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
    st = O.State(N, ph, I.TWO_PHASE)
    st.eps_p = O.to_tensor(state[6 + 6 * V:6 + 12 * V].reshape(6, N, N, N))
    st.epbar = state[6 + 12 * V:].reshape(N, N, N).copy()
    eps_np = state[6:6 + 6 * V].reshape(6, N, N, N)
    rng = np.random.default_rng(5)
    p = rng.standard_normal((6, V))
    calls = ((np.array([0, 0, 0, 0, 0, 0.0015]), fftg.FFTG_FP64, torch.float64),
             (np.array([0.001, -0.0004, 0.0002, 0.0003, 0.0, 0.0008]), fftg.FFTG_MIXED, torch.float32))
    for dE, tprec, tdt in calls:
        ref = cell.constitutive(dE=dE).cpu().numpy()
        sig = torch.full((6 * V,), np.nan, **dev)
        ep_new = torch.full((6 * V,), np.nan, **dev)
        eb_new = torch.full((V,), np.nan, **dev)
        tan = torch.full((7 * V,), np.nan, dtype=tdt, device="cuda")
        mean = np.zeros(6)
        Et = E + dE
        rc = lib.fftg_constitutive_noalloc(
            N, Et.ctypes.data_as(C.POINTER(C.c_double)), _ptr(eps), _ptr(eps_p), _ptr(epbar),
            _ptr(phase), 2, mats, tprec, _ptr(tan), _ptr(sig), _ptr(ep_new), _ptr(eb_new),
            mean.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream))
        assert rc == fftg.FFTG_OK
        got = sig.cpu().numpy()
        # against the handle call (same kernel) and the oracle
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
        res = st.constitutive(O.to_tensor(Et), O.to_tensor(eps_np))
        assert res.plastic.mean() > 0.05
        sref = O.to_comps(res.sigma).reshape(-1)
        assert np.abs(got - sref).max() <= 1e-14 * np.abs(sref).max()
        ref_mean = sref.reshape(6, V).mean(axis=1)
        assert np.abs(mean - ref_mean).max() <= 1e-14 * np.abs(ref_mean).max()
        # updated history
        epr = O.to_comps(res.eps_p).reshape(-1)
        assert np.abs(ep_new.cpu().numpy() - epr).max() <= 1e-14 * np.abs(epr).max()
        ebr = res.epbar.reshape(-1)
        assert np.abs(eb_new.cpu().numpy() - ebr).max() <= 1e-14 * np.abs(ebr).max()
        # compact tangent, in the precision asked for
        t7 = tan.double().cpu().numpy().reshape(7, V)
        assert np.isfinite(t7).all()
        cp = _apply_compact(t7, p)
        Cref = O.j2_tangent(res)
        pt = O.to_tensor(p.reshape(6, V))
        cref = O.to_comps(np.einsum("ijlmv,lmv->ijv", Cref, pt))
        scale = np.abs(Cref).max() * np.linalg.norm(p)
        tol = 1e-13 if tprec == fftg.FFTG_FP64 else 1e-6
        assert np.linalg.norm(cp - cref) <= tol * scale
    cell.close()


def test_noalloc_rejects_phase_ids_out_of_range(lib):
    N = 5
    V = N ** 3
    dev = dict(dtype=torch.float64, device="cuda")
    z6 = torch.zeros(6 * V, **dev)
    z1 = torch.zeros(V, **dev)
    sig = torch.empty(6 * V, **dev)
    ph = np.zeros(V, np.uint8)
    ph[17] = 2                                       # only phases 0 and 1 are given
    phase = torch.tensor(ph, dtype=torch.uint8, device="cuda")
    mats = (fftg.fftg_phase * 2)(*[fftg.fftg_phase(*m.as_tuple()) for m in I.TWO_PHASE])
    E = np.array([0.001, 0, 0, 0, 0, 0.0])
    mean = np.zeros(6)
    stream = torch.cuda.current_stream().cuda_stream
    args = (N, E.ctypes.data_as(C.POINTER(C.c_double)), _ptr(z6), _ptr(z6), _ptr(z1), _ptr(phase),
            2, mats, fftg.FFTG_FP64, None, _ptr(sig), None, None,
            mean.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream))
    assert lib.fftg_constitutive_noalloc(*args) == fftg.FFTG_EINVAL
    ph[17] = 1                                       # valid again: the flag starts at zero
    phase.copy_(torch.tensor(ph, dtype=torch.uint8, device="cuda"))
    assert lib.fftg_constitutive_noalloc(*args) == fftg.FFTG_OK
    assert np.isfinite(sig.cpu().numpy()).all()


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
