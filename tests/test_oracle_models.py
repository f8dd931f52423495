"""Pins of the oracle's non-linear elastic (Section 4.1) and visco-plastic
(Section 4.3) material updates.

Non-linear elasticity:
* n = 1 is linear elasticity with shear modulus sigma_0 / (3 eps_0);
* the tangent of Eq. (model:nlin-tangent) is the derivative of the stress
  (central finite difference) and has major symmetry (the model is
  hyperelastic);
* the paper's laminate (Table 2: sigma_0/G = 0.5, eps_0 = 0.1, n = 10, one
  increment to E12 = 0.05) against its one-dimensional exact solution, with
  quadratic Newton convergence (Table 3's shape).

Visco-plasticity:
* n = 1 has the closed-form dgamma = gamma_0 dt seq / (sigma_0 + 3 G gamma_0 dt);
* the returned stress satisfies Norton's rule dgamma = gamma_0 dt
  (sigma_eq / sigma_0)^(1/n), evaluated from the tensor stress itself;
* the tangent is the derivative of the update (finite difference);
* in pure shear at a constant strain rate the backward-Euler stress
  converges at first order to scipy's stiff ODE solution of the rate
  equations;
* the paper's visco-plastic laminate (Table 2: sigma_0/G = 0.1, eps_0 = 0.1,
  t_0 = 0.1, n = 0.3), loaded to E12 = 0.05 in equal time steps, against the
  same time stepping of its one-dimensional reduction (brentq per step).
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import inputs as I

G = 0.386
K = 0.833


def _sym(rng, scale):
    A = rng.standard_normal((3, 3)) * scale
    return 0.5 * (A + A.T)


def _dev(rng, scale):
    A = _sym(rng, scale)
    return A - np.trace(A) / 3.0 * np.eye(3)


def _a(v):
    return np.array([v], dtype=np.float64)


def _fd_check(update, C, eps, h=1e-7, tol=1e-6):
    for (l, m) in O.PAIRS:
        d = np.zeros((3, 3))
        if l == m:
            d[l, l] = h
        else:
            d[l, m] = d[m, l] = 0.5 * h
        fd = (update(eps + d) - update(eps - d)) / (2.0 * h)
        an = 0.5 * (C[:, :, l, m] + C[:, :, m, l])
        assert np.abs(fd - an).max() <= tol * np.abs(C).max()


# ------------------------------------------------------------ non-linear elasticity
def _nle(eps, s0=0.5 * G, e0=0.1, n=10.0, k=K):
    e = np.asarray(eps, dtype=np.float64).reshape(3, 3, 1)
    return O.nonlinear_elastic_update(e, np.zeros((3, 3, 1)), np.zeros(1), _a(k), _a(s0), _a(e0), _a(n))


def test_nle_n1_is_linear_elasticity():
    rng = np.random.default_rng(1)
    s0, e0 = 0.3, 0.05
    Gl = s0 / (3.0 * e0)
    Ce = K * O.II + 2.0 * Gl * O.I4d
    for _ in range(20):
        eps = _sym(rng, 0.01)
        r = _nle(eps, s0, e0, 1.0)
        assert np.abs(r.sigma[:, :, 0] - np.einsum("ijlm,lm->ij", Ce, eps)).max() <= 1e-15
        assert np.abs(O.nle_tangent(r)[..., 0] - Ce).max() <= 1e-14


@pytest.mark.parametrize("n", [0.5, 3.0, 10.0])
def test_nle_tangent_is_derivative_and_symmetric(n):
    rng = np.random.default_rng(int(n * 10))
    eps = _sym(rng, 0.05)
    C = O.nle_tangent(_nle(eps, n=n))[..., 0]
    _fd_check(lambda e: _nle(e, n=n).sigma[:, :, 0], C, eps)
    assert np.abs(C - C.transpose(2, 3, 0, 1)).max() <= 1e-15 * np.abs(C).max()
    assert np.abs(C - C.transpose(1, 0, 2, 3)).max() <= 1e-15 * np.abs(C).max()


def _laminate(N, n1, soft_elastic, phase1):
    return I.laminate(N, n1, axis=0), (soft_elastic, phase1)


def _quadratic(d):
    assert len(d) >= 3
    for a, b in zip(d[:-1], d[1:]):
        if a > 1e-8:
            assert b <= 10.0 * a * a


def test_paper_laminate_nonlinear_elastic():
    # pure shear e = eps_12: eps_eq = (2/sqrt3)|e|, N_12 = sign(e)/sqrt3, so
    # sigma_12 = sigma_0 (eps_eq / eps_0)^n / sqrt3 in phase 1, 2 G e in phase 2
    s0, e0, n = 0.5 * G, 0.1, 10.0
    N, n1 = 9, 3
    ph, mats = _laminate(N, n1, I.Phase(K, G, 1e9, 0.0), I.NonlinearElastic(K, s0, e0, n))
    st = O.State(N, ph, mats)
    E12 = 0.05
    r = O.solve_increment(st, np.array([0, 0, 0, 0, 0, E12]), 1e-12, 1e-14)
    assert r.converged
    f = n1 / N
    t1 = lambda e: s0 * ((2.0 / math.sqrt(3.0)) * e / e0) ** n / math.sqrt(3.0)
    F = lambda e1: t1(e1) - 2.0 * G * (E12 - f * e1) / (1.0 - f)
    e1 = brentq(F, 1e-12, E12 / f, xtol=1e-300, rtol=1e-15, maxiter=500)
    e2 = (E12 - f * e1) / (1.0 - f)
    eps12 = st.eps_star[0, 1] + st.E[0, 1]
    assert np.abs(eps12[ph == 1] - e1).max() <= 1e-10 * E12
    assert np.abs(eps12[ph == 0] - e2).max() <= 1e-10 * E12
    assert abs(r.sigma[5] - 2.0 * G * e2) <= 1e-10 * 2.0 * G * e2
    _quadratic(r.newton_norms)


# ------------------------------------------------------------ visco-plasticity
S0V, E0V, T0V = 0.1 * G, 0.1, 0.1


def _visco(eps, ep=None, eb=0.0, n=0.3, dt=1e-3, s0=S0V):
    e = np.asarray(eps, dtype=np.float64).reshape(3, 3, 1)
    ep = np.zeros((3, 3, 1)) if ep is None else np.asarray(ep).reshape(3, 3, 1)
    return O.visco_update(e, ep, _a(eb), _a(K), _a(G), _a(s0), _a(E0V), _a(T0V), _a(n), dt)


def _seq(sig):
    s = sig - np.trace(sig) / 3.0 * np.eye(3)
    return math.sqrt(1.5 * np.sum(s * s))


def test_visco_n1_closed_form():
    rng = np.random.default_rng(3)
    gdt = E0V / T0V * 1e-2
    for _ in range(20):
        seq = 0.05 * rng.random() + 1e-4
        dg = O.visco_dgamma(np.array([seq]), G, S0V, gdt, 1.0)[0]
        ref = gdt * seq / (S0V + 3.0 * G * gdt)
        assert abs(dg - ref) <= 1e-14 * ref


@pytest.mark.parametrize("n", [0.3, 1.0, 2.0])
def test_visco_update_satisfies_nortons_rule(n):
    rng = np.random.default_rng(int(10 * n))
    dt = 2e-3
    gdt = E0V / T0V * dt
    for _ in range(50):
        eps = _sym(rng, 0.02)
        ep0 = _dev(rng, 0.002)
        r = _visco(eps, ep0, 0.01, n=n, dt=dt)
        dg = r.dgamma[0]
        seq = _seq(r.sigma[:, :, 0])
        assert r.plastic[0] and dg > 0
        assert abs(dg - gdt * (seq / S0V) ** (1.0 / n)) <= 1e-12 * dg
        assert abs(np.trace(r.eps_p[:, :, 0] - ep0)) <= 1e-16


@pytest.mark.parametrize("n", [0.3, 1.0, 2.0])
def test_visco_tangent_is_derivative(n):
    rng = np.random.default_rng(7)
    eps = _sym(rng, 0.02)
    ep0 = _dev(rng, 0.002)
    r = _visco(eps, ep0, n=n)
    C = O.j2_tangent(r)[..., 0]
    _fd_check(lambda e: _visco(e, ep0, n=n).sigma[:, :, 0], C, eps)


def test_visco_backward_euler_converges_to_the_rate_equations():
    # pure shear at a constant rate: d tau/dt = 2 G (edot - sqrt3/2 gdot),
    # gdot = gamma_0 (sqrt3 |tau| / sigma_0)^(1/n)
    n, T, E12 = 0.3, 0.2, 0.05
    edot = E12 / T
    g0 = E0V / T0V

    def rhs(t, y):
        tau = y[0]
        return [2.0 * G * (edot - math.sqrt(3.0) / 2.0 * g0 * (math.sqrt(3.0) * abs(tau) / S0V) ** (1.0 / n)
                           * math.copysign(1.0, tau))]

    ref = solve_ivp(rhs, (0.0, T), [0.0], method="Radau", rtol=1e-12, atol=1e-16).y[0, -1]
    errs = []
    for k in (50, 200, 800):
        ep, eb = np.zeros((3, 3)), 0.0
        for j in range(1, k + 1):
            eps = np.zeros((3, 3)); eps[0, 1] = eps[1, 0] = E12 * j / k
            r = _visco(eps, ep, eb, n=n, dt=T / k)
            ep, eb = r.eps_p[:, :, 0], r.epbar[0]
        errs.append(abs(r.sigma[0, 1, 0] - ref))
    assert errs[2] <= 1e-3 * abs(ref)
    assert errs[1] <= 0.35 * errs[0] and errs[2] <= 0.35 * errs[1]   # first order


def test_paper_laminate_visco_plastic():
    n, k, T, E12 = 0.3, 50, 0.2, 0.05
    dt = T / k
    N, n1 = 9, 3
    ph, mats = _laminate(N, n1, I.Phase(K, G, 1e9, 0.0), I.ViscoPlastic(K, G, S0V, E0V, T0V, n))
    st = O.State(N, ph, mats, dt=dt)
    f = n1 / N
    g0dt = E0V / T0V * dt
    # one-dimensional reduction: phase 1 history (plastic shear strain p)
    p = 0.0
    for j in range(1, k + 1):
        r = O.solve_increment(st, np.array([0, 0, 0, 0, 0, E12 / k]), 1e-12, 1e-14)
        assert r.converged
        Et = E12 * j / k

        def tau1(e1):
            tt = 2.0 * G * (e1 - p)
            sq = math.sqrt(3.0) * abs(tt)
            if sq == 0.0:
                return tt, 0.0
            g = lambda x: x - g0dt * (max(sq - 3.0 * G * x, 0.0) / S0V) ** (1.0 / n)
            x = brentq(g, 0.0, sq / (3.0 * G), xtol=1e-300, rtol=1e-15, maxiter=500)
            return tt - math.copysign(math.sqrt(3.0) * G * x, tt), math.copysign(math.sqrt(3.0) / 2.0 * x, tt)

        F = lambda e1: tau1(e1)[0] - 2.0 * G * (Et - f * e1) / (1.0 - f)
        e1 = brentq(F, Et - 0.1, Et / f + 0.1, xtol=1e-300, rtol=1e-15, maxiter=500)
        p += tau1(e1)[1]
    e2 = (E12 - f * e1) / (1.0 - f)
    eps12 = st.eps_star[0, 1] + st.E[0, 1]
    assert np.abs(eps12[ph == 1] - e1).max() <= 1e-9 * E12
    assert np.abs(eps12[ph == 0] - e2).max() <= 1e-9 * E12
    assert abs(r.sigma[5] - 2.0 * G * e2) <= 1e-9 * 2.0 * G * e2


def test_kept_final_update_of_a_visco_increment_is_the_converged_stress():
    # solve_increment_keep evaluates the last stress update again against
    # the previous history: with the increment's time step (Section 4.3),
    # its stress field is the converged one, so its mean is the homogenised
    # stress of the increment and it is the elastic stress C_e : (eps -
    # eps_p) of the committed plastic strain
    N, k, T, E12 = 9, 5, 0.2, 0.05
    ph, mats = _laminate(N, 3, I.Phase(K, G, 1e9, 0.0), I.ViscoPlastic(K, G, S0V, E0V, T0V, 0.3))
    st = O.State(N, ph, mats, dt=T / k)
    for _ in range(2):
        r = O.solve_increment_keep(st, np.array([0, 0, 0, 0, 0, E12 / k]), 1e-10, 1e-12)
    sig = st.last_res.sigma
    assert np.abs(O.to_comps(sig.reshape(3, 3, -1).mean(axis=-1)) - r.sigma).max() <= 1e-13
    ee = st.eps_star + st.E[:, :, None, None, None] - st.eps_p
    tr = ee[0, 0] + ee[1, 1] + ee[2, 2]
    el = 2.0 * G * ee
    for i in range(3):
        el[i, i] += (K - 2.0 * G / 3.0) * tr
    assert np.abs(el - sig).max() <= 1e-13
