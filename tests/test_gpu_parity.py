"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances, written here and derived from the arithmetic:
* FP64 operators: the transform chain has O(log N) roundoff of ~1e-16 per
  operation; 1e-12 of the input norm leaves a factor 100 of margin.
* FP32 operators: the same chain in FP32 (unit roundoff 6e-8, about
  3 log2(N) butterfly levels): 2e-5 of the input norm.
* FP64 solver: 1e-10 relative in the homogenised stress and 1e-9 relative L2
  in the voxel strain, with identical Newton and CG counts.
* Mixed solver: the same Newton tolerance is met and the homogenised stress
  agrees with the FP64 oracle to 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_05970_gb300 import build
    build.build()
    fftg.load()


def _sym_field(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((6, N, N, N))


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda").reshape(-1)


def _cell(N, phase=None, mats=I.TWO_PHASE, precision="fp64", **kw):
    if phase is None:
        phase = np.zeros((N, N, N), np.uint8)
    return fftg.Cell(N, phase, mats, precision=precision, **kw)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


# ------------------------------------------------------------ projection
@pytest.mark.parametrize("N", [3, 5, 15, 27, 45, 75])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_projection_matches_oracle(N, prec):
    tau = _sym_field(N, N)
    dt = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        tau = tau.astype(np.float32).astype(np.float64)
    cell = _cell(N, nrhs_tangent=0)
    out = cell.project(_dev(tau, dt)).double().cpu().numpy().reshape(6, N, N, N)
    ref = O.to_comps(O.project(O.to_tensor(tau)))
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(tau)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "fp32", "dd"])
def test_projection_matches_oracle_135(prec):
    # "dd": FP64 buffers, double-float FFTs (the mixed path's residual)
    N = 135
    tau = _sym_field(N, 135)
    dt = torch.float32 if prec == "fp32" else torch.float64
    if prec == "fp32":
        tau = tau.astype(np.float32).astype(np.float64)
    cell = _cell(N, nrhs_tangent=0)
    out = cell.project(_dev(tau, dt), dd=prec == "dd").double().cpu().numpy().reshape(6, N, N, N)
    ref = O.to_comps(O.project(O.to_tensor(tau)))
    tol = 2e-5 if prec == "fp32" else 1e-12
    assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(tau)


def _plane_waves(N, nw, seed):
    """Sum of real plane waves A_w cos(2 pi k_w.x / N + phi_w) and its exact
    projection sum Ghat(k_w) : A_w cos(...) (oracle Ghat per wave)."""
    rng = np.random.default_rng(seed)
    x = np.arange(N, dtype=np.float64)
    tau = np.zeros((6, N, N, N))
    gt = np.zeros((6, N, N, N))
    for w in range(nw):
        k = rng.integers(-(N - 1) // 2, (N - 1) // 2 + 1, size=3)
        if w == 0:
            k = np.array([0, 0, 0])
        A6 = rng.standard_normal(6)
        ph = rng.uniform(0, 2 * np.pi)
        arg = (2 * np.pi / N) * (k[0] * x[:, None, None] + k[1] * x[None, :, None]
                                 + k[2] * x[None, None, :]) + ph
        cw = np.cos(arg)
        G = O.ghat(k.astype(np.float64))
        GA = O.to_comps(np.einsum("ijlm,lm->ij", G, O.to_tensor(A6)))
        for c in range(6):
            tau[c] += A6[c] * cw
            gt[c] += GA[c] * cw
    return tau, gt


@pytest.mark.parametrize("N,prec", [(243, "fp64"), (243, "fp32"), (135, "fp32")])
def test_projection_full_size_plane_waves(N, prec):
    # exact at any size: the output of a sum of Fourier modes is the sum of
    # Ghat(k) applied to each mode (the k = 0 mode is removed)
    tau, gt = _plane_waves(N, 5, 11)
    dt = torch.float64 if prec == "fp64" else torch.float32
    cell = _cell(N, nrhs_tangent=0, precision="mixed" if prec == "fp32" else "fp64")
    out = cell.project(_dev(tau, dt)).double().cpu().numpy().reshape(6, N, N, N)
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.linalg.norm(out - gt) <= tol * np.linalg.norm(tau)


# ------------------------------------------------------------ constitutive + matvec
def _plastic_state(N, seed):
    rng = np.random.default_rng(seed)
    ph, _, _ = I.random_spheres(N, 0.3, seed, r_min=1.0, r_max=3.0)
    # amplitude chosen so that 30-60 % of the voxels return plastically
    eps = 0.0015 * rng.standard_normal((6, N, N, N))
    E = np.array([0.00075, -0.000375, 0.0001875, 0.000375, -0.00075, 0.001125])
    return ph, eps, E


@pytest.mark.parametrize("N", [5, 15, 27])
def test_constitutive_matches_oracle(N):
    ph, eps, E = _plastic_state(N, 3)
    cell = _cell(N, ph, precision="fp64", nrhs_tangent=0)
    sig = cell.constitutive(dE=E, eps=_dev(eps, torch.float64)).cpu().numpy().reshape(6, N, N, N)
    st = O.State(N, ph, I.TWO_PHASE)
    res = st.constitutive(O.to_tensor(E), O.to_tensor(eps))
    assert res.plastic.mean() > 0.2 and (~res.plastic).mean() > 0.05
    ref = O.to_comps(res.sigma)
    assert np.abs(sig - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("N,prec", [(5, "fp64"), (15, "fp64"), (27, "fp64"), (45, "fp64"),
                                    (15, "fp32"), (45, "fp32")])
def test_matvec_matches_oracle(N, prec):
    ph, eps, E = _plastic_state(N, 4)
    precision = "fp64" if prec == "fp64" else "mixed"
    dt = torch.float64 if prec == "fp64" else torch.float32
    cell = _cell(N, ph, precision=precision, nrhs_tangent=0)
    cell.constitutive(dE=E, eps=_dev(eps, torch.float64))
    p = O.to_comps(O.project(O.to_tensor(_sym_field(N, 5))))
    if prec == "fp32":
        p = p.astype(np.float32).astype(np.float64)
    q, pq = cell.matvec(_dev(p, dt))
    q = q.double().cpu().numpy().reshape(6, N, N, N)
    st = O.State(N, ph, I.TWO_PHASE)
    tan = O.Tangent(st.constitutive(O.to_tensor(E), O.to_tensor(eps)))
    qr = O.matvec(tan, O.to_tensor(p))
    ref = O.to_comps(qr)
    tol = 1e-12 if prec == "fp64" else 2e-5
    # scale: ||C|| ||p|| (C = O(1), shear modulus 0.386)
    assert np.linalg.norm(q - ref) <= tol * 3.0 * np.linalg.norm(p)
    pq_ref = O.inner(O.to_tensor(p), qr)
    assert abs(pq - pq_ref) <= (1e-12 if prec == "fp64" else 1e-5) * abs(pq_ref)


# ------------------------------------------------------------ solver
def _run_oracle(w, n_inc, tol_nw, tol_cg, keep=False):
    st = O.State(w["N"], w["phase"], w["mats"])
    out = []
    for dE in w["dE"][:n_inc]:
        r = (O.solve_increment_keep if keep else O.solve_increment)(st, dE, tol_nw, tol_cg)
        out.append((r, st.eps_star.copy()))
    return st, out


def test_step_fp64_laminate15_matches_oracle_and_closed_form():
    w = I.workload("laminate15")
    st, ref = _run_oracle(w, 10, w["tol_newton"], w["tol_cg"])
    cell = _cell(15, w["phase"], w["mats"], precision="fp64")
    for i, dE in enumerate(w["dE"]):
        sig, nn, nc = cell.step(dE, w["tol_newton"], w["tol_cg"])
        r, es = ref[i]
        assert np.abs(sig - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()
        assert nn == r.newton_iters
        assert nc == r.cg_iters
        eps = cell.field(fftg.FFTG_FIELD_STRAIN)
        Et = np.sum(w["dE"][:i + 1], axis=0)
        eps_ref = O.to_comps(es) + Et[:, None, None, None]
        assert _rel(eps, eps_ref) <= 1e-9


@pytest.mark.parametrize("N,seed", [(15, 11), (27, 5)])
def test_step_fp64_spheres_matches_oracle(N, seed):
    ph, _, _ = I.random_spheres(N, 0.3, seed, r_min=2.0, r_max=4.0)
    w = dict(N=N, phase=ph, mats=I.TWO_PHASE, dE=I.shear_path(0.02, 20))
    n_inc = 4
    st, ref = _run_oracle(w, n_inc, 1e-5, 1e-8)
    cell = _cell(N, ph, precision="fp64")
    E = np.zeros(6)
    for i in range(n_inc):
        sig, nn, nc = cell.step(w["dE"][i], 1e-5, 1e-8)
        E += w["dE"][i]
        r, es = ref[i]
        assert np.abs(sig - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()
        assert (nn, nc) == (r.newton_iters, r.cg_iters)
        eps = cell.field(fftg.FFTG_FIELD_STRAIN)
        assert _rel(eps, O.to_comps(es) + E[:, None, None, None]) <= 1e-9
    s = cell.stats()
    assert s["cg_per_newton"] == ref[-1][0].cg_per_newton


def test_step_mixed_spheres_reaches_tolerance_and_matches():
    N = 27
    ph, _, _ = I.random_spheres(N, 0.3, 5, r_min=2.0, r_max=4.0)
    w = dict(N=N, phase=ph, mats=I.TWO_PHASE, dE=I.shear_path(0.02, 20))
    st, ref = _run_oracle(w, 4, 1e-5, 1e-8)
    cell = _cell(N, ph, precision="mixed")
    for i in range(4):
        sig, nn, nc = cell.step(w["dE"][i], 1e-5, 1e-8)
        r, _ = ref[i]
        assert np.abs(sig - r.sigma).max() <= 1e-6 * np.abs(r.sigma).max()
        s = cell.stats()
        assert s["newton_norm"][-1] <= 1e-5 or s["newton_norm"][-1] == 0.0


@pytest.mark.slow
def test_mixed_vs_fp64_spheres135_shear():
    # 135^3, random spheres (r in [3, 8], hard fraction 0.3), pure shear in
    # increments of 0.001: the FP32-inner path reaches the same Newton
    # tolerance and its homogenised stress agrees with the FP64 path (itself
    # oracle-exact at smaller sizes) to 1e-6
    w = I.workload("spheres135", seed=2)
    c64 = _cell(135, w["phase"], w["mats"], precision="fp64", nrhs_tangent=0)
    c32 = _cell(135, w["phase"], w["mats"], precision="mixed", nrhs_tangent=0)
    for dE in w["dE"][:4]:
        s64, _, _ = c64.step(dE, 1e-5, 1e-8)
        s32, _, _ = c32.step(dE, 1e-5, 1e-8)
        assert np.abs(s32 - s64).max() <= 1e-6 * np.abs(s64).max()
        st = c32.stats()
        assert st["newton_norm"][-1] <= 1e-5
    c64.close()
    c32.close()


def test_tangent_matches_oracle():
    w = I.workload("laminate15")
    st = O.State(15, w["phase"], w["mats"])
    for dE in w["dE"][:2]:
        O.solve_increment(st, dE, 1e-10, 1e-12)
    O.solve_increment_keep(st, w["dE"][2], 1e-10, 1e-12)
    Cref = O.macro_tangent(st, 1e-12)
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-5)):
        cell = _cell(15, w["phase"], w["mats"], precision=prec)
        for dE in w["dE"][:3]:
            cell.step(dE, 1e-10, 1e-12)
        C, _ = cell.tangent(1e-12)
        assert np.abs(C - Cref).max() <= tol * np.abs(Cref).max(), prec


def test_fixed_iteration_mode_matches_oracle():
    N = 15
    ph, _, _ = I.random_spheres(N, 0.3, 11, r_min=2.0, r_max=4.0)
    st = O.State(N, ph, I.TWO_PHASE)
    cell = _cell(N, ph, precision="fp64", fixed_cg=7, fixed_newton=2)
    for dE in I.shear_path(0.02, 20)[:3]:
        r = O.solve_increment(st, dE, 1e-5, 1e-8, fixed_cg=7, fixed_newton=2)
        sig, nn, nc = cell.step(dE, 1e-5, 1e-8)
        assert nn == 2 and nn == r.newton_iters
        assert np.abs(sig - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()


# ------------------------------------------------------------ boundary behaviour
def test_state_roundtrip_and_errors():
    N = 15
    w = I.workload("laminate15")
    cell = _cell(N, w["phase"], w["mats"], precision="fp64")
    with pytest.raises(fftg.FftgError) as e:
        cell.tangent(1e-8)
    assert e.value.code == fftg.FFTG_ESTATE
    for dE in w["dE"][:3]:
        cell.step(dE, 1e-5, 1e-8)
    s = cell.get_state()
    sig_a, _, _ = cell.step(w["dE"][3], 1e-5, 1e-8)
    cell.set_state(s)
    sig_b, _, _ = cell.step(w["dE"][3], 1e-5, 1e-8)
    assert np.array_equal(sig_a, sig_b)
    # NaN increment: rejected, committed state unchanged
    snap = cell.get_state()
    with pytest.raises(fftg.FftgError) as e:
        cell.step([np.nan, 0, 0, 0, 0, 0], 1e-5, 1e-8)
    assert e.value.code == fftg.FFTG_ENAN
    assert np.array_equal(cell.get_state(), snap)
    # Newton cap: fails without committing
    c2 = _cell(N, w["phase"], w["mats"], precision="fp64", max_newton=1)
    for dE in w["dE"][:1]:
        c2.step(dE, 1e-5, 1e-8)
    before = c2.get_state()
    with pytest.raises(fftg.FftgError) as e:
        c2.step(w["dE"][1] * 5, 1e-12, 1e-8)
    assert e.value.code == fftg.FFTG_ENOCONV_NEWTON
    assert np.array_equal(c2.get_state(), before)
    with pytest.raises(fftg.FftgError):
        fftg.Cell(15, np.full((15, 15, 15), 3, np.uint8), I.TWO_PHASE)


def test_stress_field_and_homogenised_stress_agree():
    w = I.workload("laminate15")
    cell = _cell(15, w["phase"], w["mats"], precision="fp64")
    for dE in w["dE"][:4]:
        sig, _, _ = cell.step(dE, 1e-5, 1e-8)
    S = cell.field(fftg.FFTG_FIELD_STRESS)
    assert np.abs(S.reshape(6, -1).mean(axis=1) - sig).max() <= 1e-15
    C, _ = cell.tangent(1e-8)  # the tangent survives the field read
    assert np.all(np.isfinite(C))


def test_mixed_path_stays_on_the_fp64_solution_over_a_long_path():
    # 20 increments of the shear path on a 27^3 sphere cell: each FP32 inner
    # solution is projected onto compatible fields, so no incompatible strain
    # accumulates in eps* and the mixed path tracks the FP64 one (without the
    # projection the homogenised stresses drifted apart to 1e-4)
    N = 27
    ph, _, _ = I.random_spheres(N, 0.3, 5, r_min=2.0, r_max=4.0)
    c64 = _cell(N, ph, precision="fp64", nrhs_tangent=0)
    c32 = _cell(N, ph, precision="mixed", nrhs_tangent=0)
    for dE in I.shear_path(0.02, 20):
        s64, _, _ = c64.step(dE, 1e-5, 1e-8)
        s32, _, _ = c32.step(dE, 1e-5, 1e-8)
        assert np.abs(s32 - s64).max() <= 1e-7 * np.abs(s64).max()
    e64 = c64.field(fftg.FFTG_FIELD_STRAIN)
    e32 = c32.field(fftg.FFTG_FIELD_STRAIN)
    assert _rel(e32, e64) <= 1e-6
    c64.close()
    c32.close()
