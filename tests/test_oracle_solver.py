"""Pins of the oracle's Newton-CG solver against exact solutions.

* two-phase laminates have piecewise-constant exact solutions that follow
  from traction continuity and compatibility across the interface (the
  paper reproduces them "with two elements", Section 5.1, and observes no
  artefact at the nodes);
* the plastic laminate with equal elasticity reduces to a scalar
  pure-shear problem per phase with a closed-form response;
* a homogeneous cell needs no fluctuation and no CG iteration;
* with a homogeneous isotropic tangent, G C has two distinct eigenvalues on
  compatible fields, so CG ends in two iterations;
* the macroscopic tangent equals a central finite difference of the solver;
* Newton with the consistent tangent converges quadratically once the
  plastic set settles (the shape of Table 3).
"""
import math

import numpy as np
import pytest

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import inputs as I


def _tau_phase(g, ph):
    """Pure-shear response of one J2 phase, g = engineering shear strain."""
    if ph.G * g <= ph.sigma_y / math.sqrt(3.0):
        return ph.G * g
    return (ph.sigma_y / math.sqrt(3.0) + ph.H * g / 3.0) / (1.0 + ph.H / (3.0 * ph.G))


def _laminate_closed_form(E12, f_h, hard, soft):
    """Solve tau_h(g_h) = tau_s(g_s), f_h g_h + f_s g_s = 2 E12 by bisection."""
    f_s = 1.0 - f_h
    lo, hi = 0.0, 2.0 * E12 / f_h
    for _ in range(200):
        gh = 0.5 * (lo + hi)
        gs = (2.0 * E12 - f_h * gh) / f_s
        if _tau_phase(gh, hard) - _tau_phase(gs, soft) > 0.0:
            hi = gh
        else:
            lo = gh
    gh = 0.5 * (lo + hi)
    gs = (2.0 * E12 - f_h * gh) / f_s
    return _tau_phase(gh, hard), gh / 2.0, gs / 2.0


def test_plastic_laminate_matches_closed_form_every_increment():
    w = I.workload("laminate15")
    st = O.State(w["N"], w["phase"], w["mats"])
    soft, hard = w["mats"]
    E12 = 0.0
    ph = w["phase"]
    for dE in w["dE"]:
        E12 += dE[5]
        r = O.solve_increment(st, dE, w["tol_newton"], w["tol_cg"])
        assert r.converged
        tau, e_h, e_s = _laminate_closed_form(E12, 5.0 / 15.0, hard, soft)
        assert abs(r.sigma[5] - tau) <= 1e-9 * tau
        assert np.abs(r.sigma[:5]).max() <= 1e-12
        eps12 = st.eps_star[0, 1] + E12
        assert np.abs(eps12[ph == 1] - e_h).max() <= 1e-9 * E12
        assert np.abs(eps12[ph == 0] - e_s).max() <= 1e-9 * E12
        # the hard phase stays elastic along the whole path
        assert st.epbar[ph == 1].max() == 0.0


def _elastic_laminate_exact(E, f_a, A, B):
    """Exact strains of a laminate with interface normal e1, isotropic phases.

    Components not involving index 1 equal E in both phases; the jumps
    d = (d11, d12, d13) in eps_1j make sigma_1j continuous, with
    eps^a = E + f_b d and eps^b = E - f_a d on those components.
    """
    f_b = 1.0 - f_a

    def sig(eps, ph):
        lam = ph.K - 2.0 * ph.G / 3.0
        return lam * np.trace(eps) * np.eye(3) + 2.0 * ph.G * eps

    def strains(d):
        ea, eb = E.copy(), E.copy()
        for j in range(3):
            ea[0, j] += f_b * d[j]; eb[0, j] -= f_a * d[j]
            if j:
                ea[j, 0] = ea[0, j]; eb[j, 0] = eb[0, j]
        return ea, eb

    def jump(d):
        ea, eb = strains(d)
        return sig(ea, A)[0] - sig(eb, B)[0]

    j0 = jump(np.zeros(3))
    M = np.stack([jump(np.eye(3)[k]) - j0 for k in range(3)], axis=1)
    d = np.linalg.solve(M, -j0)
    return strains(d), sig(strains(d)[0], A), sig(strains(d)[1], B)


def test_elastic_laminate_contrast_exact_and_one_newton_step():
    soft = I.Phase(0.833, 0.386, 1e9, 0.0)
    hard = I.Phase(8.33, 3.86, 1e9, 0.0)
    N = 15
    ph = I.laminate(N, 5, axis=0)
    st = O.State(N, ph, (soft, hard))
    dE = np.array([0.01, 0.002, -0.003, 0.001, 0.002, 0.004])
    r = O.solve_increment(st, dE, 1e-10, 1e-13)
    (ea, eb), sa, sb = _elastic_laminate_exact(O.to_tensor(dE), 5.0 / 15.0, hard, soft)
    eps = st.eps_star + st.E[:, :, None, None, None]
    scale = np.abs(ea).max()
    assert np.abs(eps[:, :, ph == 1] - ea[:, :, None]).max() <= 1e-10 * scale
    assert np.abs(eps[:, :, ph == 0] - eb[:, :, None]).max() <= 1e-10 * scale
    Sig = O.to_comps((5.0 * sa + 10.0 * sb) / 15.0)
    assert np.abs(r.sigma - Sig).max() <= 1e-10 * np.abs(Sig).max()
    # linear problem: the first Newton step is the solution
    assert r.newton_iters <= 2 and r.newton_norms[-1] <= 1e-10


def test_homogeneous_cell_has_no_fluctuation():
    N = 9
    st = O.State(N, np.zeros((N, N, N), np.uint8), (I.SOFT,))
    dE = np.array([0.001, -0.0005, 0.0002, 0.0, 0.0007, 0.002])
    for _ in range(3):
        r = O.solve_increment(st, dE, 1e-8, 1e-10)
        assert r.cg_iters == 0 and r.newton_iters == 1
        assert np.abs(st.eps_star).max() == 0.0
    # homogeneous J2 along a proportional path: compare with the single-point
    # update driven through the same increments
    ep = np.zeros((3, 3, 1)); eb = np.zeros(1); E = np.zeros((3, 3))
    for _ in range(3):
        E = E + O.to_tensor(dE)
        one = O.j2_update(E.reshape(3, 3, 1), ep, eb, *(np.array([v]) for v in I.SOFT.as_tuple()[:5]))
        ep, eb = one.eps_p, one.epbar
    assert np.abs(r.sigma - O.to_comps(one.sigma[:, :, 0])).max() <= 1e-16


def test_cg_two_iterations_for_homogeneous_isotropic_tangent():
    N = 9
    st = O.State(N, np.zeros((N, N, N), np.uint8), (I.Phase(2.0, 0.7, 1e9, 0.0),))
    res = st.constitutive(np.zeros((3, 3)), np.zeros((3, 3, N, N, N)))
    tan = O.Tangent(res)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 3, N, N, N)); x = x + x.transpose(1, 0, 2, 3, 4)
    b = O.project(x)
    sol, it, rel = O.cg(lambda p: O.matvec(tan, p), b, 1e-13, 50)
    assert it <= 2 and rel <= 1e-13
    chk = O.matvec(tan, sol) - b
    assert np.sqrt(O.inner(chk, chk) / O.inner(b, b)) <= 1e-12


def test_macro_tangent_matches_finite_difference_and_is_symmetric():
    w = I.workload("laminate15")
    soft, hard = w["mats"]
    st0 = O.State(w["N"], w["phase"], w["mats"])
    for dE in w["dE"][:2]:
        O.solve_increment(st0, dE, 1e-10, 1e-12)
    dE = w["dE"][2]
    snap = (st0.E.copy(), st0.eps_star.copy(), st0.eps_p.copy(), st0.epbar.copy())

    def fresh():
        return O.State(w["N"], w["phase"], w["mats"], E=snap[0].copy(),
                       eps_star=snap[1].copy(), eps_p=snap[2].copy(), epbar=snap[3].copy())

    st = fresh()
    O.solve_increment_keep(st, dE, 1e-10, 1e-12)
    C = O.macro_tangent(st, 1e-12)
    h = 1e-7
    fd = np.zeros((6, 6))
    for j in range(6):
        e = np.zeros(6); e[j] = h
        sp = O.solve_increment(fresh(), dE + e, 1e-11, 1e-12).sigma
        sm = O.solve_increment(fresh(), dE - e, 1e-11, 1e-12).sigma
        fd[:, j] = (sp - sm) / (2.0 * h)
    assert np.abs(C - fd).max() <= 1e-6 * np.abs(C).max()
    assert np.abs(C - C.T).max() <= 1e-8 * np.abs(C).max()


def test_macro_tangent_homogeneous_elastic_convention():
    # column j perturbs tensor component j (shears symmetric): the 12,12
    # entry of an isotropic elastic cell is 2G, not G
    N = 5
    ph = I.Phase(1.3, 0.4, 1e9, 0.0)
    st = O.State(N, np.zeros((N, N, N), np.uint8), (ph,))
    O.solve_increment_keep(st, np.array([1e-4, 0, 0, 0, 0, 0]), 1e-8, 1e-10)
    C = O.macro_tangent(st, 1e-12)
    lam = ph.K - 2 * ph.G / 3
    ref = np.zeros((6, 6))
    ref[:3, :3] = lam
    ref[[0, 1, 2], [0, 1, 2]] += 2 * ph.G
    ref[[3, 4, 5], [3, 4, 5]] = 2 * ph.G
    assert np.abs(C - ref).max() <= 1e-13


def test_newton_quadratic_once_plastic_set_settles():
    ph, _, _ = I.random_spheres(15, 0.3, 11, r_min=2.0, r_max=4.0)
    st = O.State(15, ph, I.TWO_PHASE)
    for _ in range(2):
        O.solve_increment(st, [0, 0, 0, 0, 0, 0.001], 1e-5, 1e-8)
    r = O.solve_increment(st, [0, 0, 0, 0, 0, 0.001], 1e-8, 1e-10)
    nn = r.newton_norms
    assert r.converged and nn[-1] <= 1e-8
    # the last two steps: quadratic (a linear rate of 0.1 would fail this)
    assert nn[-1] <= 200.0 * nn[-2] ** 2
    assert nn[-2] <= 200.0 * nn[-3] ** 2


def test_increment_same_with_textbook_fft(monkeypatch):
    # the whole Newton-CG increment with the textbook mixed-radix FFT in
    # place of the library FFT: the same iteration counts, and the
    # homogenised stress and the strain field within the tolerances of the
    # FP64 parity tests (1e-10 and 1e-9: a different rounding of each FFT,
    # carried through the CG recursions)
    N = 9
    ph, _, _ = I.random_spheres(N, 0.3, 7, r_min=1.5, r_max=3.0)
    out = {}
    for impl in ("library", "textbook"):
        monkeypatch.setattr(O, "FFT_IMPL", impl)
        st = O.State(N, ph, I.TWO_PHASE)
        rs = [O.solve_increment(st, dE, 1e-6, 1e-8) for dE in I.shear_path(0.006, 3)[:2]]
        out[impl] = (rs, st.eps_star.copy())
    (ra, ea), (rb, eb) = out["library"], out["textbook"]
    assert any(r.cg_iters > 0 for r in ra)
    for a, b in zip(ra, rb):
        assert (a.newton_iters, a.cg_iters) == (b.newton_iters, b.cg_iters)
        assert np.abs(a.sigma - b.sigma).max() <= 1e-10 * np.abs(a.sigma).max()
    assert np.linalg.norm(ea - eb) <= 1e-9 * np.linalg.norm(ea)
