"""Pins of the finite-strain oracle (the extension named in Section 6: F in
place of the strain, first Piola-Kirchhoff stress, gradient projection).

Checked against what the mathematics fixes, not against the oracle itself:
* Ghat_fs is the orthogonal projector onto gradient fields at each
  frequency: symmetric, idempotent, identity on a (x) xi, zero when A xi = 0;
* on a grid, G leaves the gradient of a band-limited periodic displacement
  unchanged (written analytically) and removes a constant and a field whose
  rows are divergence free (the equilibrium fields);
* St. Venant-Kirchhoff: P is the derivative of the energy W and K that of P
  (central differences), K has the major symmetry of a hyperelastic
  tangent, P(R F) = R P(F) for a rotation R;
* a homogeneous cell keeps F* = 0 and gives P(Fbar);
* a laminate matches the closed-form two-layer solution (continuity of
  P e1 across the layers, solved by scipy), including a large deformation;
* the small-strain limit is the pinned small-strain oracle with
  K = lambda + 2 mu/3, G = mu, with an error that falls linearly with the
  load;
* Newton with this tangent converges quadratically;
* the 9x9 macroscopic tangent equals the local tangent for a homogeneous
  cell, the central differences of full solves (and is major-symmetric, as
  the Hessian of the homogenised energy), and the derivative of the
  laminate's closed form.
"""
import numpy as np
import pytest
from scipy.optimize import fsolve

from oracle import fftg_finite_strain as FS
from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import inputs as I

LAM0, MU0 = I.SVK_SOFT.lam, I.SVK_SOFT.mu


def _rotation(axis, angle):
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


# ------------------------------------------------------------------ projector
def test_ghat_fs_is_the_orthogonal_projector_onto_gradients():
    rng = np.random.default_rng(1)
    for _ in range(20):
        xi = rng.integers(-6, 7, size=3).astype(float)
        if not xi.any():
            continue
        G = FS.ghat_fs(xi)
        M = G.reshape(9, 9)
        assert np.abs(M - M.T).max() <= 1e-15
        assert np.abs(M @ M - M).max() <= 1e-14
        a = rng.standard_normal(3)
        grad = np.outer(a, xi)
        assert np.abs(np.einsum("ijlm,lm->ij", G, grad) - grad).max() <= 1e-13 * np.abs(grad).max()
        # rows orthogonal to xi (A xi = 0) are removed
        B = rng.standard_normal((3, 3))
        B -= np.outer(B @ xi, xi) / (xi @ xi)
        assert np.abs(np.einsum("ijlm,lm->ij", G, B)).max() <= 1e-14
        assert abs(np.trace(M) - 3.0) <= 1e-14      # rank 3: one vector per row
    assert not FS.ghat_fs((0.0, 0.0, 0.0)).any()


def _waves(N):
    x = np.arange(N, dtype=float)
    return np.meshgrid(x, x, x, indexing="ij")


def test_projection_keeps_gradients_and_removes_equilibrium_fields():
    N = 9
    X = _waves(N)
    rng = np.random.default_rng(2)
    grad = np.zeros((3, 3, N, N, N))
    div_free = np.zeros((3, 3, N, N, N))
    for xi in ((1, 0, 0), (0, 2, -1), (3, 1, 4), (-2, 2, 1)):
        xi = np.array(xi, float)
        ph = 2 * np.pi * (xi[0] * X[0] + xi[1] * X[1] + xi[2] * X[2]) / N
        a = rng.standard_normal(3)
        # u_i = a_i sin(2 pi xi.x / N): grad u_ij = a_i (2 pi xi_j / N) cos(...)
        grad += np.einsum("i,j,...->ij...", a, 2 * np.pi * xi / N, np.cos(ph))
        # W_ij = b_i c_j sin(...), c . xi = 0: every row divergence free
        c = rng.standard_normal(3)
        c -= (c @ xi) / (xi @ xi) * xi
        b = rng.standard_normal(3)
        div_free += np.einsum("i,j,...->ij...", b, c, np.sin(ph))
    const = rng.standard_normal((3, 3))[:, :, None, None, None] * np.ones((1, 1, N, N, N))
    out = FS.project_fs(grad + div_free + const)
    assert np.abs(out - grad).max() <= 1e-13 * np.abs(grad).max()


def test_projection_is_not_the_small_strain_one():
    # a (x) e1 with a along e2 is a gradient, but its symmetric part is a
    # small-strain compatible field only together with its transpose
    N = 9
    X = _waves(N)
    A = np.zeros((3, 3, N, N, N))
    A[1, 0] = np.cos(2 * np.pi * X[0] / N)
    assert np.abs(FS.project_fs(A) - A).max() <= 1e-14
    At = np.zeros_like(A)
    At[0, 1] = A[1, 0]                       # the transpose: rows along e2 only
    assert np.abs(FS.project_fs(At)).max() <= 1e-14


# ------------------------------------------------------------------- material
def _random_F(rng, scale=0.3):
    return np.eye(3) + scale * rng.standard_normal((3, 3))


def test_svk_stress_is_the_derivative_of_the_energy():
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(5):
        F = _random_F(rng)
        P = FS.svk_update(F, LAM0, MU0).P
        dW = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                e = np.zeros((3, 3))
                e[i, j] = h
                dW[i, j] = (FS.svk_energy(F + e, LAM0, MU0) - FS.svk_energy(F - e, LAM0, MU0)) / (2 * h)
        assert np.abs(dW - P).max() <= 1e-8 * np.abs(P).max()


def test_svk_tangent_is_the_derivative_of_the_stress():
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(5):
        F = _random_F(rng)
        res = FS.svk_update(F[:, :, None], np.array([LAM0]), np.array([MU0]))
        K = FS.svk_tangent(res)[..., 0]
        Kfd = np.zeros((3, 3, 3, 3))
        for k in range(3):
            for l in range(3):
                e = np.zeros((3, 3))
                e[k, l] = h
                Kfd[:, :, k, l] = (FS.svk_update(F + e, LAM0, MU0).P - FS.svk_update(F - e, LAM0, MU0).P) / (2 * h)
        assert np.abs(K - Kfd).max() <= 1e-8 * np.abs(K).max()
        M = K.reshape(9, 9)
        assert np.abs(M - M.T).max() <= 1e-14 * np.abs(M).max()   # major symmetry


def test_svk_is_objective():
    rng = np.random.default_rng(5)
    for _ in range(5):
        F = _random_F(rng)
        R = _rotation(rng.standard_normal(3), rng.uniform(0, np.pi))
        P = FS.svk_update(F, LAM0, MU0).P
        assert np.abs(FS.svk_update(R @ F, LAM0, MU0).P - R @ P).max() <= 1e-14 * np.abs(P).max()


def test_svk_at_identity_is_isotropic_small_strain_elasticity():
    res = FS.svk_update(np.eye(3)[:, :, None], np.array([LAM0]), np.array([MU0]))
    K = FS.svk_tangent(res)[..., 0]
    K_iso = LAM0 * np.einsum("ij,kl->ijkl", np.eye(3), np.eye(3)) + MU0 * (
        np.einsum("ik,jl->ijkl", np.eye(3), np.eye(3)) + np.einsum("il,jk->ijkl", np.eye(3), np.eye(3)))
    assert np.abs(K - K_iso).max() <= 1e-15


# -------------------------------------------------------------------- solver
def test_homogeneous_cell_keeps_zero_fluctuation():
    N = 5
    st = FS.State(N, np.zeros((N, N, N), np.uint8), (I.SVK_SOFT.as_tuple(),))
    dF = np.array([[0.2, 0.1, 0.0], [0.0, -0.1, 0.05], [0.03, 0.0, 0.1]])
    r = FS.solve_increment(st, dF, 1e-10, 1e-12)
    assert r.converged
    assert np.abs(st.Fstar).max() <= 1e-14
    P = FS.svk_update(np.eye(3) + dF, LAM0, MU0).P
    assert np.abs(r.P - P).max() <= 1e-14 * np.abs(P).max()


def _laminate_closed_form(Fbar, f_hard, hard, soft):
    """Two layers normal to e1: F_k = Fbar + a_k (x) e1, f_h a_h + f_s a_s = 0,
    P(F_h) e1 = P(F_s) e1. Returns the volume average of P."""
    def P_of(a, m):
        return FS.svk_update(Fbar + np.outer(a, [1.0, 0.0, 0.0]), m.lam, m.mu).P

    def resid(a_h):
        a_s = -f_hard / (1.0 - f_hard) * a_h
        return (P_of(a_h, hard) - P_of(a_s, soft))[:, 0]

    a_h = fsolve(resid, np.zeros(3), xtol=1e-15)
    assert np.abs(resid(a_h)).max() <= 1e-13
    a_s = -f_hard / (1.0 - f_hard) * a_h
    return f_hard * P_of(a_h, hard) + (1.0 - f_hard) * P_of(a_s, soft)


@pytest.mark.parametrize("scale", [0.01, 0.3])
def test_laminate_matches_the_closed_form(scale):
    N, n_hard = 9, 4
    ph = I.laminate(N, n_hard, axis=0)
    st = FS.State(N, ph, tuple(m.as_tuple() for m in I.SVK_TWO_PHASE))
    dF = scale * np.array([[0.5, 0.4, -0.2], [0.3, -0.2, 0.25], [0.1, 0.35, 0.2]])
    r = FS.solve_increment(st, dF, 1e-12, 1e-12)
    assert r.converged
    P = _laminate_closed_form(np.eye(3) + dF, n_hard / N, I.SVK_HARD, I.SVK_SOFT)
    assert np.abs(r.P - P).max() <= 1e-11 * np.abs(P).max()


def test_small_strain_limit_is_the_small_strain_oracle():
    N = 9
    ph, _, _ = I.random_spheres(N, 0.3, 7, r_min=1.5, r_max=3.0)
    mats_fs = tuple(m.as_tuple() for m in I.SVK_TWO_PHASE)
    mats_ss = tuple(I.Phase(m.lam + 2.0 * m.mu / 3.0, m.mu, 1e12, 0.0) for m in I.SVK_TWO_PHASE)
    H6 = np.array([0.4, -0.1, 0.2, 0.3, -0.25, 0.5])
    H = O.to_tensor(H6)
    errs = []
    for t in (1e-3, 1e-4):
        st = FS.State(N, ph, mats_fs)
        r = FS.solve_increment(st, t * H, 1e-12, 1e-12)
        ss = O.State(N, ph, mats_ss)
        s = O.solve_increment(ss, t * H6, 1e-12, 1e-12)
        sig = O.to_tensor(s.sigma)
        errs.append(np.abs(r.P - sig).max() / np.abs(sig).max())
    assert errs[0] <= 1e-2 and errs[1] <= 1e-3
    assert 5.0 <= errs[0] / errs[1] <= 20.0            # first order in the load


def test_newton_converges_quadratically():
    N = 9
    ph, _, _ = I.random_spheres(N, 0.3, 7, r_min=1.5, r_max=3.0)
    st = FS.State(N, ph, tuple(m.as_tuple() for m in I.SVK_TWO_PHASE))
    dF = np.array([[0.15, 0.1, 0.0], [0.05, -0.08, 0.1], [0.0, 0.12, 0.06]])
    r = FS.solve_increment(st, dF, 1e-13, 1e-14)
    assert r.converged
    n = r.newton_norms
    assert len(n) >= 4
    # in the quadratic regime each norm is at most a modest multiple of the
    # square of the previous one
    for a, b in zip(n[1:-1], n[2:]):
        if a < 1e-2 and b > 1e-13:
            assert b <= 50.0 * a * a


def test_solution_is_objective():
    N = 9
    ph, _, _ = I.random_spheres(N, 0.3, 11, r_min=1.5, r_max=3.0)
    mats = tuple(m.as_tuple() for m in I.SVK_TWO_PHASE)
    Fbar = np.eye(3) + np.array([[0.1, 0.05, 0.0], [0.02, -0.05, 0.04], [0.0, 0.06, 0.08]])
    R = _rotation((1.0, 2.0, -0.5), 0.7)
    out = []
    for Fb in (Fbar, R @ Fbar):
        st = FS.State(N, ph, mats)
        out.append(FS.solve_increment(st, Fb - np.eye(3), 1e-12, 1e-12).P)
    assert np.abs(out[1] - R @ out[0]).max() <= 1e-10 * np.abs(out[0]).max()


# ------------------------------------------------------------ macro tangent
def test_macro_tangent_of_a_homogeneous_cell_is_the_local_tangent():
    N = 5
    st = FS.State(N, np.zeros((N, N, N), np.uint8), (I.SVK_SOFT.as_tuple(),))
    dF = np.array([[0.2, 0.1, 0.0], [0.0, -0.1, 0.05], [0.03, 0.0, 0.1]])
    FS.solve_increment(st, dF, 1e-12, 1e-12)
    C, n = FS.macro_tangent(st, 1e-12)
    res = FS.svk_update((np.eye(3) + dF)[:, :, None], np.array([LAM0]), np.array([MU0]))
    K = FS.svk_tangent(res)[..., 0].reshape(9, 9)
    assert np.abs(C - K).max() <= 1e-13 * np.abs(K).max() and n == 0


def test_macro_tangent_is_the_derivative_of_the_homogenised_stress():
    # central differences of full solves: dPbar/dFbar_kl
    N = 9
    ph, _, _ = I.random_spheres(N, 0.3, 7, r_min=1.5, r_max=3.0)
    mats = tuple(m.as_tuple() for m in I.SVK_TWO_PHASE)
    dF = np.array([[0.08, 0.05, 0.0], [0.02, -0.04, 0.03], [0.0, 0.04, 0.03]])
    st = FS.State(N, ph, mats)
    FS.solve_increment(st, dF, 1e-13, 1e-14)
    C, _ = FS.macro_tangent(st, 1e-12)
    h = 1e-5
    Cfd = np.zeros((9, 9))
    for col in range(9):
        E = np.zeros((3, 3))
        E[col // 3, col % 3] = h
        Pp = FS.solve_increment(FS.State(N, ph, mats, Fbar=st.Fbar.copy(), Fstar=st.Fstar.copy()), E, 1e-13, 1e-14).P
        Pm = FS.solve_increment(FS.State(N, ph, mats, Fbar=st.Fbar.copy(), Fstar=st.Fstar.copy()), -E, 1e-13, 1e-14).P
        Cfd[:, col] = ((Pp - Pm) / (2 * h)).reshape(9)
    assert np.abs(C - Cfd).max() <= 1e-6 * np.abs(C).max()
    # major symmetry of the homogenised hyperelastic tangent
    assert np.abs(C - C.T).max() <= 1e-9 * np.abs(C).max()


def test_macro_tangent_of_the_laminate_matches_the_closed_form():
    N, n_hard = 9, 4
    ph = I.laminate(N, n_hard, axis=0)
    st = FS.State(N, ph, tuple(m.as_tuple() for m in I.SVK_TWO_PHASE))
    dF = 0.2 * np.array([[0.5, 0.4, -0.2], [0.3, -0.2, 0.25], [0.1, 0.35, 0.2]])
    FS.solve_increment(st, dF, 1e-13, 1e-14)
    C, _ = FS.macro_tangent(st, 1e-13)
    h = 1e-6
    f = n_hard / N
    Cfd = np.zeros((9, 9))
    for col in range(9):
        E = np.zeros((3, 3))
        E[col // 3, col % 3] = h
        Cfd[:, col] = ((_laminate_closed_form(np.eye(3) + dF + E, f, I.SVK_HARD, I.SVK_SOFT)
                        - _laminate_closed_form(np.eye(3) + dF - E, f, I.SVK_HARD, I.SVK_SOFT)) / (2 * h)).reshape(9)
    assert np.abs(C - Cfd).max() <= 1e-6 * np.abs(C).max()


def test_ghat_fs_row_form():
    # The fused finite-strain P3 takes row i of Ghat_fs : A as (A_i . n) n,
    # n = xi / |xi|: the oracle's delta_il xi_j xi_m / |xi|^2 contracted
    # with A_lm, for complex A and any xi != 0.
    rng = np.random.default_rng(22)
    for _ in range(50):
        xi = rng.integers(-121, 122, size=3).astype(np.float64)
        if not xi.any():
            continue
        A = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        ref = np.einsum("ijlm,lm->ij", FS.ghat_fs(xi), A)
        n = xi / np.linalg.norm(xi)
        got = np.outer(A @ n, n)
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(A).max()
        assert np.abs(np.outer(n, A @ n) - ref).max() > 1e-6 * np.abs(ref).max()  # the transpose is not it
