"""Pins of the oracle's basic scheme (Section 3.2: Richardson's iteration
with the reference medium C_ref = (lambda_min + lambda_max)/2 I_s).

Checked against:
* Appendix A's reference-medium Green operator computed through the acoustic
  tensor: Gamma_ref for C_ref = c I_s equals Ghat / c (so the scheme is
  Richardson's iteration on G D with the step 1/c);
* the eigenvalues of the elastic tangent, 3K (once) and 2G (five times);
* the contraction bound of Richardson's iteration with the optimal step,
  ||r_k|| <= ((kappa - 1)/(kappa + 1))^k ||r_0||, kappa = lambda_max/lambda_min;
* the same increment solution as CG;
* the iteration growth the paper states: linear in the contrast for the
  basic scheme, about its square root for CG.
"""
import numpy as np
import pytest

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import inputs as I


def test_gamma_ref_of_scaled_identity_is_ghat_over_c():
    rng = np.random.default_rng(0)
    Is = 0.5 * (np.einsum("il,jm->ijlm", np.eye(3), np.eye(3)) +
                np.einsum("im,jl->ijlm", np.eye(3), np.eye(3)))
    for _ in range(20):
        xi = rng.integers(-7, 8, size=3).astype(float)
        if not xi.any():
            continue
        c = 0.1 + 5.0 * rng.random()
        assert np.abs(O.gamma_ref(xi, c * Is) - O.ghat(xi) / c).max() <= 1e-14 / c


def test_bounds_of_the_elastic_tangent():
    N = 5
    K, G = 0.9, 0.35
    st = O.State(N, np.zeros((N, N, N), np.uint8), (I.Phase(K, G, 1e9, 0.0),))
    res = st.constitutive(np.zeros((3, 3)), np.zeros((3, 3, N, N, N)))
    ev = np.linalg.eigvalsh(np.moveaxis(O.mandel(O.point_tangent(res, slice(0, 1))), -1, 0))[0]
    assert np.allclose(np.sort(ev), [2 * G] * 5 + [3 * K], rtol=1e-14)
    lo, hi = O.tangent_bounds(res)
    assert abs(lo - min(2 * G, 3 * K)) <= 1e-14 and abs(hi - max(2 * G, 3 * K)) <= 1e-14


def _elastic_spheres(N, contrast, seed=3):
    ph, _, _ = I.random_spheres(N, 0.3, seed, r_min=1.0, r_max=2.5)
    soft = I.Phase(0.833, 0.386, 1e9, 0.0)
    hard = I.Phase(0.833 * contrast, 0.386 * contrast, 1e9, 0.0)
    return ph, (soft, hard)


def test_richardson_contracts_at_the_optimal_rate():
    N = 15
    ph, mats = _elastic_spheres(N, 10.0)
    st = O.State(N, ph, mats)
    E = O.to_tensor(np.array([0.001, 0.0, -0.0005, 0.0, 0.0, 0.002]))
    res = st.constitutive(E, np.zeros((3, 3, N, N, N)))
    tan = O.Tangent(res)
    b = -O.project(res.sigma)
    lo, hi = O.tangent_bounds(res)
    rate = (hi / lo - 1.0) / (hi / lo + 1.0)
    omega = 2.0 / (lo + hi)
    x = np.zeros_like(b)
    r0 = np.sqrt(O.inner(b, b))
    for k in range(1, 30):
        x += omega * (b - O.matvec(tan, x))
        r = np.sqrt(O.inner(b - O.matvec(tan, x), b - O.matvec(tan, x)))
        assert r <= rate ** k * r0 * (1.0 + 1e-9)


def test_richardson_and_cg_give_the_same_increment():
    N = 9
    ph, _, _ = I.random_spheres(N, 0.3, 5, r_min=1.5, r_max=3.0)
    out = {}
    for solver in ("cg", "richardson"):
        st = O.State(N, ph, I.TWO_PHASE)
        for dE in I.shear_path(0.0045, 3):     # plastic from the second increment
            r = O.solve_increment(st, dE, 1e-9, 1e-11, max_cg=20000, solver=solver)
            assert r.converged
        assert r.cg_iters > 0 and st.epbar.max() > 0
        out[solver] = (r.sigma, st.eps_star.copy())
    assert np.abs(out["cg"][0] - out["richardson"][0]).max() <= 1e-9 * np.abs(out["cg"][0]).max()
    assert np.abs(out["cg"][1] - out["richardson"][1]).max() <= 1e-8 * np.abs(out["cg"][1]).max()


def test_iterations_grow_with_the_contrast_as_the_paper_states():
    N = 9
    E = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.001])
    its = {}
    for contrast in (10.0, 100.0):
        ph, mats = _elastic_spheres(N, contrast)
        for solver in ("cg", "richardson"):
            st = O.State(N, ph, mats)
            r = O.solve_increment(st, E, 1e-6, 1e-8, max_cg=20000, solver=solver)
            its[(solver, contrast)] = r.cg_iters
    rich = its[("richardson", 100.0)] / its[("richardson", 10.0)]
    cg = its[("cg", 100.0)] / its[("cg", 10.0)]
    assert rich > 5.0          # ~ kappa: a factor of about 10
    assert cg < 4.0            # ~ sqrt(kappa): a factor of about 3
    assert its[("richardson", 100.0)] > 10 * its[("cg", 100.0)]
