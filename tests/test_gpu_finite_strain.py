"""The finite-strain path on the GPU (include/fftg_fs.h) against the
finite-strain oracle, element by element, and against properties that hold
at any size.

Tolerances: FP64 operators 1e-12 of the largest entry (FFT rounding only);
FP64 increments 1e-10 in the homogenised stress with identical Newton and CG
counts (the oracle and the kernels round differently, and the solver's
stopping tests sit well away from their thresholds); mixed precision 1e-6
(the Newton tolerance; the FP64 residual makes Newton an iterative
refinement of the FP32 inner solves).
"""
import numpy as np
import pytest

from oracle import fftg_finite_strain as FS
from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MATS = tuple(m.as_tuple() for m in I.SVK_TWO_PHASE)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_05970_gb300 import build
    build.build()
    fftg.load()


def _path(n_inc, scale=1.0):
    """A mixed stretch-shear path of n_inc equal increments of dF."""
    G = np.array([[0.06, 0.08, 0.0], [0.02, -0.03, 0.05], [0.0, 0.04, 0.03]])
    return [scale * G / n_inc] * n_inc


def _spheres(N, seed=5):
    ph, _, _ = I.random_spheres(N, 0.3, seed, r_min=max(1.5, N / 9), r_max=max(3.0, N / 4))
    return ph


@pytest.mark.parametrize("N", [3, 15, 25, 45, 75, 81])
def test_projection_matches_the_oracle(N):
    rng = np.random.default_rng(N)
    A = rng.standard_normal((3, 3, N, N, N))
    ref = FS.project_fs(A)
    cell64 = fftg.FsCell(N, np.zeros((N, N, N), np.uint8), MATS[:1], precision="fp64")
    out = cell64.project(torch.tensor(A.reshape(-1), device="cuda")).cpu().numpy().reshape(A.shape)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    cell64.close()
    cell32 = fftg.FsCell(N, np.zeros((N, N, N), np.uint8), MATS[:1], precision="mixed")
    out = cell32.project(torch.tensor(A.reshape(-1), dtype=torch.float32, device="cuda"))
    out = out.cpu().double().numpy().reshape(A.shape)
    assert np.abs(out - ref).max() <= 2e-6 * np.abs(ref).max()
    cell32.close()


def test_projection_is_idempotent_and_keeps_gradients():
    N = 27
    x = np.arange(N, dtype=float)
    X = np.meshgrid(x, x, x, indexing="ij")
    xi = np.array([2.0, -1.0, 3.0])
    ph = 2 * np.pi * (xi[0] * X[0] + xi[1] * X[1] + xi[2] * X[2]) / N
    a = np.array([0.3, -0.2, 0.5])
    grad = np.einsum("i,j,...->ij...", a, 2 * np.pi * xi / N, np.cos(ph))
    cell = fftg.FsCell(N, np.zeros((N, N, N), np.uint8), MATS[:1], precision="fp64")
    g = cell.project(torch.tensor(grad.reshape(-1), device="cuda"))
    assert np.abs(g.cpu().numpy().reshape(grad.shape) - grad).max() <= 1e-13
    rng = np.random.default_rng(1)
    A = torch.tensor(rng.standard_normal(9 * N ** 3), device="cuda")
    GA = cell.project(A)
    assert (cell.project(GA) - GA).abs().max().item() <= 1e-13 * GA.abs().max().item()
    cell.close()


def test_matvec_matches_the_oracle_at_a_deformed_state():
    N = 15
    ph = _spheres(N)
    cell = fftg.FsCell(N, ph, MATS, precision="fp64")
    for dF in _path(2):
        cell.step(dF, 1e-10, 1e-12)
    F = cell.field(fftg.FFTG_FS_FIELD_DEFGRAD)
    st = FS.State(N, ph, MATS)
    res = FS.svk_update(F, st.lam, st.mu)
    rng = np.random.default_rng(2)
    p = rng.standard_normal((3, 3, N, N, N))
    ref = FS.project_fs(FS.Tangent(res).apply(p))
    q, pq = cell.matvec(torch.tensor(p.reshape(-1), device="cuda"))
    q = q.cpu().numpy().reshape(p.shape)
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(pq - FS.inner(p, ref)) <= 1e-12 * abs(FS.inner(p, ref))
    # the committed stress field
    P = cell.field(fftg.FFTG_FS_FIELD_STRESS)
    assert np.abs(P - res.P).max() <= 1e-14 * np.abs(res.P).max()
    cell.close()


@pytest.mark.parametrize("N", [9, 25])
def test_fp64_increments_match_the_oracle(N):
    ph = _spheres(N)
    st = FS.State(N, ph, MATS)
    cell = fftg.FsCell(N, ph, MATS, precision="fp64")
    for dF in _path(3, 2.0):
        r = FS.solve_increment(st, dF, 1e-9, 1e-11)
        P, nn, nc = cell.step(dF, 1e-9, 1e-11)
        assert r.converged
        assert np.abs(P - r.P).max() <= 1e-10 * np.abs(r.P).max()
        assert (nn, nc) == (r.newton_iters, r.cg_iters)
        s = cell.stats()
        assert s["cg_per_newton"] == r.cg_per_newton
        assert np.allclose(s["residual"], r.residual, rtol=1e-6, atol=1e-13)
    F = cell.field(fftg.FFTG_FS_FIELD_DEFGRAD)
    assert np.abs(F - (st.Fstar + st.Fbar[:, :, None, None, None])).max() <= 1e-10
    cell.close()


def test_mixed_increments_reach_the_fp64_result():
    N = 15
    ph = _spheres(N, seed=8)
    st = FS.State(N, ph, MATS)
    cell = fftg.FsCell(N, ph, MATS, precision="mixed")
    for dF in _path(3, 2.0):
        r = FS.solve_increment(st, dF, 1e-8, 1e-10)
        P, nn, nc = cell.step(dF, 1e-7, 1e-8)
        assert cell.stats()["newton_norm"][-1] <= 1e-7
        assert np.abs(P - r.P).max() <= 1e-6 * np.abs(r.P).max()
    cell.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_laminate_matches_the_closed_form(precision, tol):
    from scipy.optimize import fsolve
    N, n_hard = 45, 17
    ph = I.laminate(N, n_hard, axis=0)
    dF = 0.3 * np.array([[0.5, 0.4, -0.2], [0.3, -0.2, 0.25], [0.1, 0.35, 0.2]])
    Fbar = np.eye(3) + dF
    f = n_hard / N
    hard, soft = I.SVK_HARD, I.SVK_SOFT

    def P_of(a, m):
        return FS.svk_update(Fbar + np.outer(a, [1.0, 0.0, 0.0]), m.lam, m.mu).P

    def resid(a_h):
        return (P_of(a_h, hard) - P_of(-f / (1 - f) * a_h, soft))[:, 0]

    a_h = fsolve(resid, np.zeros(3), xtol=1e-15)
    P_ref = f * P_of(a_h, hard) + (1 - f) * P_of(-f / (1 - f) * a_h, soft)
    cell = fftg.FsCell(N, ph, MATS, precision=precision)
    P, nn, nc = cell.step(dF, 1e-10 if precision == "fp64" else 1e-8, 1e-12 if precision == "fp64" else 1e-8)
    assert np.abs(P - P_ref).max() <= tol * np.abs(P_ref).max()
    cell.close()


def test_zero_increment_and_homogeneous_cell():
    N = 27
    cell = fftg.FsCell(N, np.zeros((N, N, N), np.uint8), MATS[:1], precision="mixed")
    P, nn, nc = cell.step(np.zeros((3, 3)), 1e-8, 1e-8)
    assert np.abs(P).max() == 0.0 and nc == 0
    dF = np.array([[0.2, 0.1, 0.0], [0.0, -0.1, 0.05], [0.03, 0.0, 0.1]])
    P, nn, nc = cell.step(dF, 1e-8, 1e-8)
    ref = FS.svk_update(np.eye(3) + dF, *MATS[0]).P
    assert np.abs(P - ref).max() <= 1e-14 * np.abs(ref).max()
    assert nc == 0
    cell.close()


def test_failed_increment_leaves_the_state_unchanged():
    N = 9
    ph = _spheres(N)
    cell = fftg.FsCell(N, ph, MATS, precision="fp64", max_newton=1)
    F0 = cell.field(fftg.FFTG_FS_FIELD_DEFGRAD)
    with pytest.raises(fftg.FftgError) as e:
        cell.step(_path(1)[0], 1e-12, 1e-12)
    assert e.value.code == fftg.FFTG_ENOCONV_NEWTON
    assert np.array_equal(cell.field(fftg.FFTG_FS_FIELD_DEFGRAD), F0)
    cell.close()


def _equilibrium_defect(P):
    """max over xi != 0 of |Phat(xi) xi| / (|xi| max|Phat|): zero exactly when
    every row of P is divergence free in the trigonometric sense, i.e.
    G P = 0 (computed with numpy's FFT from the definition)."""
    N = P.shape[-1]
    Ph = np.fft.fftn(P, axes=(2, 3, 4))
    k = np.fft.fftfreq(N) * N
    xi = np.stack(np.meshgrid(k, k, k, indexing="ij"))
    nrm = np.sqrt(np.sum(xi * xi, axis=0))
    nrm[0, 0, 0] = 1.0
    d = np.einsum("ij...,j...->i...", Ph, xi) / nrm
    Ph[:, :, 0, 0, 0] = 0.0
    return np.abs(d).max() / np.abs(Ph).max()


def test_converged_state_is_in_equilibrium_at_243():
    # the workload and launch configuration of the finite-strain bench line
    w = I.workload("fs_spheres243")
    N, ph = w["N"], w["phase"]
    cell = fftg.FsCell(N, ph, w["mats"], precision="mixed")
    for dF in w["dF"][:2]:
        P, nn, nc = cell.step(dF, w["tol_newton"], w["tol_cg"])
        assert cell.stats()["newton_norm"][-1] <= w["tol_newton"]
    Pf = cell.field(fftg.FFTG_FS_FIELD_STRESS)
    assert np.abs(Pf.reshape(3, 3, -1).mean(axis=-1) - P).max() <= 1e-12 * np.abs(P).max()
    # sampled voxels: P from the committed F by the oracle's material law
    F = cell.field(fftg.FFTG_FS_FIELD_DEFGRAD)
    cell.close()
    rng = np.random.default_rng(0)
    idx = tuple(rng.integers(0, N, size=(3, 256)))
    lam = np.array([m.lam for m in w["mats"]])[ph[idx]]
    mu = np.array([m.mu for m in w["mats"]])[ph[idx]]
    Ps = FS.svk_update(F[(slice(None), slice(None)) + idx], lam, mu).P
    assert np.abs(Ps - Pf[(slice(None), slice(None)) + idx]).max() <= 1e-13 * np.abs(Ps).max()
    # the mean of F is Fbar: F* has no mean (to the FP32 rounding of the
    # projected corrections)
    Fbar = np.eye(3) + w["dF"][:2].sum(axis=0)
    assert np.abs(F.reshape(3, 3, -1).mean(axis=-1) - Fbar).max() <= 1e-8
    del F
    assert _equilibrium_defect(Pf) <= 1e-5


# ------------------------------------------------------------ macro tangent
def test_fp64_macro_tangent_matches_the_oracle():
    N = 9
    ph = _spheres(N)
    st = FS.State(N, ph, MATS)
    cell = fftg.FsCell(N, ph, MATS, precision="fp64")
    for dF in _path(2, 2.0):
        FS.solve_increment(st, dF, 1e-10, 1e-12)
        cell.step(dF, 1e-10, 1e-12)
    Cref, nref = FS.macro_tangent(st, 1e-11)
    C, n = cell.tangent(1e-11)
    assert np.abs(C - Cref).max() <= 1e-9 * np.abs(Cref).max()
    assert n == nref
    cell.close()


def test_mixed_macro_tangent_reaches_the_fp64_result():
    N = 15
    ph = _spheres(N, seed=8)
    st = FS.State(N, ph, MATS)
    cell = fftg.FsCell(N, ph, MATS, precision="mixed")
    for dF in _path(2, 2.0):
        FS.solve_increment(st, dF, 1e-10, 1e-12)
        cell.step(dF, 1e-8, 1e-8)
    Cref, _ = FS.macro_tangent(st, 1e-11)
    C, n = cell.tangent(1e-8)
    assert np.abs(C - Cref).max() <= 1e-5 * np.abs(Cref).max()
    cell.close()


def test_macro_tangent_of_a_homogeneous_cell_is_the_local_tangent():
    N = 27
    cell = fftg.FsCell(N, np.zeros((N, N, N), np.uint8), MATS[:1], precision="mixed")
    dF = np.array([[0.2, 0.1, 0.0], [0.0, -0.1, 0.05], [0.03, 0.0, 0.1]])
    cell.step(dF, 1e-8, 1e-8)
    C, n = cell.tangent(1e-8)
    res = FS.svk_update((np.eye(3) + dF)[:, :, None], np.array([MATS[0][0]]), np.array([MATS[0][1]]))
    K = FS.svk_tangent(res)[..., 0].reshape(9, 9)
    assert n == 0
    assert np.abs(C - K).max() <= 1e-6 * np.abs(K).max()
    cell.close()


def test_macro_tangent_at_243_is_symmetric_and_stiff_in_stretch():
    # the bench workload: the homogenised tangent of a hyperelastic cell is
    # the Hessian of its effective energy (major-symmetric). On symmetric
    # perturbations it is positive definite at these moderate strains; the
    # three rotational directions carry only the geometric stiffness of the
    # stress (eigenvalues of the order of |P|, of either sign)
    w = I.workload("fs_spheres243")
    cell = fftg.FsCell(w["N"], w["phase"], w["mats"], precision="mixed")
    P, _, _ = cell.step(w["dF"][0], w["tol_newton"], w["tol_cg"])
    C, n = cell.tangent(w["tol_cg"])
    cell.close()
    assert n > 0
    assert np.abs(C - C.T).max() <= 1e-4 * np.abs(C).max()
    Q = np.zeros((9, 6))          # orthonormal basis of symmetric 3x3 tensors
    for c, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))):
        E = np.zeros((3, 3))
        E[i, j] = E[j, i] = 1.0
        Q[:, c] = E.reshape(9) / np.linalg.norm(E)
    ev_sym = np.linalg.eigvalsh(Q.T @ (0.5 * (C + C.T)) @ Q)
    assert ev_sym.min() > 0.1 * ev_sym.max()
    ev = np.linalg.eigvalsh(0.5 * (C + C.T))
    assert np.sort(np.abs(ev))[:3].max() <= 2.0 * np.abs(P).max()


def test_checkpoint_and_restore_continue_bit_for_bit():
    N = 15
    ph = _spheres(N)
    a = fftg.FsCell(N, ph, MATS, precision="mixed")
    path = _path(3, 2.0)
    for dF in path[:2]:
        a.step(dF, 1e-8, 1e-8)
    state = a.get_state()
    assert state.size == 9 + 9 * N ** 3
    b = fftg.FsCell(N, ph, MATS, precision="mixed")
    bad = state.copy()
    bad[100] = np.nan
    with pytest.raises(fftg.FftgError):
        b.set_state(bad)
    b.set_state(state)
    Pa, na, ca = a.step(path[2], 1e-8, 1e-8)
    Pb, nb, cb = b.step(path[2], 1e-8, 1e-8)
    assert np.array_equal(Pa, Pb) and (na, ca) == (nb, cb)
    assert np.array_equal(a.field(fftg.FFTG_FS_FIELD_DEFGRAD), b.field(fftg.FFTG_FS_FIELD_DEFGRAD))
    a.close()
    b.close()


def test_mixed_long_path_stays_on_the_oracle():
    # ten increments to F11 = 1.3 (F12 = 0.15): the FP32 inner solves must
    # not let the mixed state drift from the FP64 solution
    N = 15
    ph = _spheres(N, seed=4)
    st = FS.State(N, ph, MATS)
    cell = fftg.FsCell(N, ph, MATS, precision="mixed")
    worst = 0.0
    for dF in 3.0 * I.stretch_shear_path(10):
        r = FS.solve_increment(st, dF, 1e-9, 1e-11)
        P, nn, nc = cell.step(dF, 1e-8, 1e-8)
        assert r.converged
        worst = max(worst, np.abs(P - r.P).max() / np.abs(r.P).max())
    F = cell.field(fftg.FFTG_FS_FIELD_DEFGRAD)
    Fo = st.Fstar + st.Fbar[:, :, None, None, None]
    assert worst <= 1e-7
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo - np.eye(3)[:, :, None, None, None]) <= 1e-6
    cell.close()
