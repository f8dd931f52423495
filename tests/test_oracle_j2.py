"""Pins of the oracle's J2 return mapping (Section 4.2, n = 1).

Checked against: yield consistency after the return, the elastic branch,
a central finite difference of the stress update (the consistent tangent is
its derivative), plastic incompressibility, and the closed-form pure-shear
response of linear isotropic hardening.
"""
import math

import numpy as np
import pytest

from oracle import fftg_oracle as O

K, G, SY, H = 0.833, 0.386, 0.003, 0.01


def _one(eps, eps_p=None, epbar=0.0, k=K, g=G, sy=SY, h=H):
    eps = np.asarray(eps, dtype=np.float64).reshape(3, 3, 1)
    eps_p = np.zeros((3, 3, 1)) if eps_p is None else np.asarray(eps_p).reshape(3, 3, 1)
    a = lambda v: np.array([v], dtype=np.float64)
    return O.j2_update(eps, eps_p, a(epbar), a(k), a(g), a(sy), a(h))


def _sym(rng, scale):
    A = rng.standard_normal((3, 3)) * scale
    return 0.5 * (A + A.T)


def _seq(sig):
    s = sig - np.trace(sig) / 3.0 * np.eye(3)
    return math.sqrt(1.5 * np.sum(s * s))


def test_yield_consistency_and_incompressibility():
    rng = np.random.default_rng(0)
    n_pl = 0
    for _ in range(200):
        eps = _sym(rng, 0.02)
        ep0 = _sym(rng, 0.002)
        ep0 -= np.trace(ep0) / 3.0 * np.eye(3)
        eb0 = abs(rng.standard_normal()) * 0.01
        r = _one(eps, ep0, eb0)
        sig = r.sigma[:, :, 0]
        if r.plastic[0]:
            n_pl += 1
            phi = _seq(sig) - (SY + H * r.epbar[0])
            assert abs(phi) <= 1e-12 * SY
        else:
            assert _seq(sig) - (SY + H * eb0) <= 1e-12 * SY
        assert abs(np.trace(r.eps_p[:, :, 0])) < 1e-15
        assert r.epbar[0] >= eb0
    assert n_pl > 100


def test_elastic_branch_gives_elastic_tangent():
    eps = np.diag([1e-4, -2e-4, 5e-5])
    eps[0, 1] = eps[1, 0] = 1e-4
    r = _one(eps)
    assert not r.plastic[0]
    C = O.j2_tangent(r)[..., 0]
    Ce = K * O.II + 2.0 * G * O.I4d
    assert np.abs(C - Ce).max() == 0.0
    assert np.allclose(r.sigma[:, :, 0], np.einsum("ijlm,lm->ij", Ce, eps), atol=1e-18)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_tangent_is_derivative_of_stress_update(seed):
    rng = np.random.default_rng(seed)
    eps = _sym(rng, 0.01)
    ep0 = _sym(rng, 0.001)
    ep0 -= np.trace(ep0) / 3.0 * np.eye(3)
    eb0 = 0.004
    r = _one(eps, ep0, eb0)
    assert r.plastic[0]
    C = O.j2_tangent(r)[..., 0]
    h = 1e-7
    for (l, m) in O.PAIRS:
        d = np.zeros((3, 3))
        if l == m:
            d[l, l] = h
        else:
            d[l, m] = d[m, l] = 0.5 * h
        sp = _one(eps + d, ep0, eb0).sigma[:, :, 0]
        sm = _one(eps - d, ep0, eb0).sigma[:, :, 0]
        fd = (sp - sm) / (2.0 * h)
        an = 0.5 * (C[:, :, l, m] + C[:, :, m, l])
        assert np.abs(fd - an).max() <= 1e-6 * np.abs(C).max()


def test_pure_shear_linear_hardening_closed_form():
    # monotone pure shear: tau = G g while G g <= sigma0/sqrt3, else
    # tau = (sigma0/sqrt3 + H g / 3) / (1 + H / (3G)), g = 2 eps12
    ep = np.zeros((3, 3))
    eb = 0.0
    for g in np.linspace(0.0, 0.05, 51)[1:]:
        eps = np.zeros((3, 3)); eps[0, 1] = eps[1, 0] = g / 2
        r = _one(eps, ep, eb)
        ep = r.eps_p[:, :, 0]; eb = r.epbar[0]
        tau = r.sigma[0, 1, 0]
        if G * g <= SY / math.sqrt(3):
            ref = G * g
        else:
            ref = (SY / math.sqrt(3) + H * g / 3.0) / (1.0 + H / (3.0 * G))
        assert abs(tau - ref) <= 1e-13 * abs(ref)
        # only the 12 shear stress is non-zero
        mask = np.ones((3, 3), bool); mask[0, 1] = mask[1, 0] = False
        assert np.abs(r.sigma[:, :, 0][mask]).max() < 1e-16


def test_tangent_major_and_minor_symmetry():
    rng = np.random.default_rng(5)
    r = _one(_sym(rng, 0.02))
    assert r.plastic[0]
    C = O.j2_tangent(r)[..., 0]
    assert np.abs(C - C.transpose(1, 0, 2, 3)).max() < 1e-16
    assert np.abs(C - C.transpose(2, 3, 0, 1)).max() < 1e-15
