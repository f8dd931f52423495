"""Pins of the oracle's J2 return mapping with power-law hardening
sigma_0 + H epbar^n (Section 4.2, n != 1).

Checked against:
* the closed form dgamma = Phi_tr / (3G + H) at n = 1 (the textbook case the
  scalar solver must reduce to);
* scipy's brentq on the paper's scalar return equation (a library root
  finder in place of the oracle's bracketed Newton);
* yield consistency of the returned tensor stress, evaluated from the yield
  function itself, and plastic incompressibility;
* a central finite difference of the stress update (the consistent tangent
  with the slope n H (epbar_t + dgamma)^(n-1) is its derivative);
* path independence of the radial return on a proportional path (1, 7 or 40
  increments give the same state);
* the paper's elasto-plastic laminate (Table 2: H/G = 0.05, sigma_0/G = 0.01,
  n = 0.1, one increment to E12 = 0.05) against its exact one-dimensional
  solution: both phases in pure shear with equal sigma_12, solved by brentq;
  and quadratic convergence of the Newton iteration on it (Table 3).
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import inputs as I

K, G = 0.833, 0.386


def _one(eps, eps_p, epbar, sy, h, n, k=K, g=G):
    eps = np.asarray(eps, dtype=np.float64).reshape(3, 3, 1)
    eps_p = np.asarray(eps_p, dtype=np.float64).reshape(3, 3, 1)
    a = lambda v: np.array([v], dtype=np.float64)
    return O.j2_update(eps, eps_p, a(epbar), a(k), a(g), a(sy), a(h), a(n))


def _sym(rng, scale):
    A = rng.standard_normal((3, 3)) * scale
    return 0.5 * (A + A.T)


def _dev(rng, scale):
    A = _sym(rng, scale)
    return A - np.trace(A) / 3.0 * np.eye(3)


def _seq(sig):
    s = sig - np.trace(sig) / 3.0 * np.eye(3)
    return math.sqrt(1.5 * np.sum(s * s))


def test_scalar_return_reduces_to_closed_form_at_n_1():
    rng = np.random.default_rng(11)
    seq = 0.01 + 0.02 * rng.random(50)
    eb = 0.01 * rng.random(50)
    sy, h = 0.003, 0.01
    phi = seq - (sy + h * eb)
    dg = O.power_law_dgamma(seq, eb, G, sy, h, 1.0)
    assert np.abs(dg - phi / (3.0 * G + h)).max() <= 1e-15 * np.abs(phi / (3.0 * G)).max()


@pytest.mark.parametrize("n", [0.1, 0.3, 0.5, 2.0, 3.0])
def test_scalar_return_matches_brentq(n):
    rng = np.random.default_rng(int(10 * n))
    sy, h = 0.003, 0.05 * G
    for _ in range(40):
        eb = 0.02 * rng.random() if rng.random() < 0.7 else 0.0
        phi_tr = 0.02 * rng.random() + 1e-7
        seq = phi_tr + sy + h * eb ** n
        f = lambda x: seq - 3.0 * G * x - sy - h * (eb + x) ** n
        ref = brentq(f, 0.0, phi_tr / (3.0 * G), xtol=1e-300, rtol=1e-15, maxiter=500)
        got = O.power_law_dgamma(np.array([seq]), np.array([eb]), G, sy, h, n)[0]
        assert abs(got - ref) <= 1e-13 * ref


@pytest.mark.parametrize("n", [0.1, 0.5, 2.0])
def test_yield_consistency_and_incompressibility(n):
    rng = np.random.default_rng(7)
    sy, h = 0.003, 0.05 * G
    n_pl = 0
    for _ in range(150):
        eps = _sym(rng, 0.02)
        ep0 = _dev(rng, 0.002)
        eb0 = abs(rng.standard_normal()) * 0.01 if rng.random() < 0.8 else 0.0
        r = _one(eps, ep0, eb0, sy, h, n)
        sig = r.sigma[:, :, 0]
        if r.plastic[0]:
            n_pl += 1
            phi = _seq(sig) - (sy + h * r.epbar[0] ** n)
            assert abs(phi) <= 1e-12 * sy
            assert r.epbar[0] > eb0
        else:
            assert _seq(sig) - (sy + h * eb0 ** n) <= 1e-12 * sy
        assert abs(np.trace(r.eps_p[:, :, 0])) < 1e-15
    assert n_pl > 80


@pytest.mark.parametrize("n,eb0", [(0.1, 0.004), (0.1, 0.0), (0.5, 0.002), (2.0, 0.01)])
def test_tangent_is_derivative_of_stress_update(n, eb0):
    rng = np.random.default_rng(3)
    sy, h = 0.003, 0.05 * G
    eps = _sym(rng, 0.01)
    ep0 = _dev(rng, 0.001)
    r = _one(eps, ep0, eb0, sy, h, n)
    assert r.plastic[0]
    C = O.j2_tangent(r)[..., 0]
    step = 1e-7
    for (l, m) in O.PAIRS:
        d = np.zeros((3, 3))
        if l == m:
            d[l, l] = step
        else:
            d[l, m] = d[m, l] = 0.5 * step
        sp = _one(eps + d, ep0, eb0, sy, h, n).sigma[:, :, 0]
        sm = _one(eps - d, ep0, eb0, sy, h, n).sigma[:, :, 0]
        fd = (sp - sm) / (2.0 * step)
        an = 0.5 * (C[:, :, l, m] + C[:, :, m, l])
        assert np.abs(fd - an).max() <= 1e-6 * np.abs(C).max()


@pytest.mark.parametrize("n", [0.1, 0.3, 2.0])
def test_radial_return_is_exact_on_a_proportional_path(n):
    rng = np.random.default_rng(5)
    sy, h = 0.003, 0.05 * G
    target = _dev(rng, 0.02) + 0.002 * np.eye(3)
    out = []
    for k in (1, 7, 40):
        ep, eb = np.zeros((3, 3)), 0.0
        for j in range(1, k + 1):
            r = _one(target * j / k, ep, eb, sy, h, n)
            ep, eb = r.eps_p[:, :, 0], r.epbar[0]
        out.append((r.sigma[:, :, 0], eb))
    for sig, eb in out[1:]:
        assert np.abs(sig - out[0][0]).max() <= 1e-11 * np.abs(out[0][0]).max()
        assert abs(eb - out[0][1]) <= 1e-11 * out[0][1]


def _shear_stress_virgin(e12, sy, h, n):
    """sigma_12 of a virgin J2 point driven in one step to pure shear e12
    (the scalar return equation of Section 4.2 in pure shear, where
    sigma_eq = sqrt(3) |sigma_12| and N_12 = sqrt(3)/2 sign)."""
    t_tr = 2.0 * G * e12
    phi = math.sqrt(3.0) * abs(t_tr) - sy
    if phi <= 0.0:
        return t_tr
    f = lambda x: math.sqrt(3.0) * abs(t_tr) - 3.0 * G * x - sy - h * x ** n
    dg = brentq(f, 0.0, phi / (3.0 * G), xtol=1e-300, rtol=1e-15, maxiter=500)
    return t_tr - math.copysign(math.sqrt(3.0) * G * dg, t_tr)


def test_paper_laminate_table2_exact_and_quadratic_newton():
    # phase 1: elasto-plastic (Table 2); phase 2: linear elastic, same moduli
    sy, h, n = 0.01 * G, 0.05 * G, 0.1
    pl = I.Phase(K, G, sy, h, n)
    el = I.Phase(K, G, 1e9, 0.0)
    N, n1 = 15, 5
    ph = I.laminate(N, n1, axis=0)
    st = O.State(N, ph, (el, pl))
    E12 = 0.05
    r = O.solve_increment(st, np.array([0, 0, 0, 0, 0, E12]), 1e-12, 1e-14)
    assert r.converged
    f = n1 / N
    # exact laminate: f e1 + (1 - f) e2 = E12, sigma12(e1) = 2 G e2
    F = lambda e1: _shear_stress_virgin(e1, sy, h, n) - 2.0 * G * (E12 - f * e1) / (1.0 - f)
    e1 = brentq(F, E12, E12 / f, xtol=1e-300, rtol=1e-15, maxiter=500)
    e2 = (E12 - f * e1) / (1.0 - f)
    eps12 = st.eps_star[0, 1] + st.E[0, 1]
    assert np.abs(eps12[ph == 1] - e1).max() <= 1e-10 * E12
    assert np.abs(eps12[ph == 0] - e2).max() <= 1e-10 * E12
    assert abs(r.sigma[5] - 2.0 * G * e2) <= 1e-10 * 2.0 * G * e2
    assert np.abs(r.sigma[:5]).max() <= 1e-12 * abs(r.sigma[5])
    # Newton converges quadratically (the shape of the paper's Table 3)
    d = r.newton_norms
    assert len(d) >= 3
    for a, b in zip(d[:-1], d[1:]):
        if a > 1e-8:
            assert b <= 10.0 * a * a
