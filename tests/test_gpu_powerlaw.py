"""Parity of the CUDA J2 kernel with power-law hardening sigma_0 + H epbar^n
(Section 4.2, n != 1) with the FP64 oracle, through the C-ABI.

Tolerances as in the other parity tests: FP64 pointwise 1e-13 of the
largest stress, FP64 operators 1e-12 and FP32 operators 2e-5 of the input
norm, FP64 solves 1e-10 in the homogenised stress with identical Newton and
CG counts, mixed solves 1e-6.

The history states are set through fftg_set_state so that both signs of
the N(x)N coefficient of the consistent tangent occur (the positive one
only for n > 1, stored with a negative K in the compact tangent).
"""

import numpy as np
import pytest

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G = 0.386
# soft phase: the paper's elasto-plastic law (Table 2 ratios, n = 0.1);
# hard phase: strong hardening with n = 3 (positive N(x)N coefficients)
PL = (I.Phase(0.833, G, 0.003, 0.05 * G, 0.1), I.Phase(0.833, G, 0.006, 20.0 * G, 3.0))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_05970_gb300 import build
    build.build()
    fftg.load()


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda").reshape(-1)


def _history(N, seed):
    rng = np.random.default_rng(seed)
    ph, _, _ = I.random_spheres(N, 0.4, seed, r_min=1.0, r_max=3.0)
    E = np.array([0.004, -0.002, 0.001, 0.003, -0.002, 0.005])
    eps = 0.02 * rng.standard_normal((6, N, N, N))
    ep = 0.002 * rng.standard_normal((6, N, N, N))
    ep[:3] -= ep[:3].mean(axis=0, keepdims=True)      # deviatoric plastic strain
    eb = 0.1 * rng.random((N, N, N))
    eb[rng.random((N, N, N)) < 0.2] = 0.0             # some virgin points
    return ph, E, eps, ep, eb


def _oracle_state(N, ph, E, eps, ep, eb):
    st = O.State(N, ph, PL)
    st.eps_p = O.to_tensor(ep)
    st.epbar = eb.copy()
    return st, st.constitutive(O.to_tensor(E), O.to_tensor(eps))


@pytest.mark.parametrize("N", [5, 15])
def test_constitutive_powerlaw_matches_oracle(N):
    ph, E, eps, ep, eb = _history(N, 21)
    cell = fftg.Cell(N, ph, PL, precision="fp64", nrhs_tangent=0)
    cell.set_state(np.concatenate([E, np.zeros(6 * N ** 3), ep.ravel(), eb.ravel()]))
    sig = cell.constitutive(eps=_dev(eps, torch.float64)).cpu().numpy().reshape(6, N, N, N)
    st, res = _oracle_state(N, ph, E, eps, ep, eb)
    assert res.plastic.mean() > 0.3
    ref = O.to_comps(res.sigma)
    assert np.abs(sig - ref).max() <= 1e-13 * np.abs(ref).max()
    cell.close()


@pytest.mark.parametrize("N,prec", [(15, "fp64"), (15, "fp32"), (27, "fp64")])
def test_matvec_powerlaw_both_tangent_signs(N, prec):
    ph, E, eps, ep, eb = _history(N, 22)
    precision = "fp64" if prec == "fp64" else "mixed"
    dt = torch.float64 if prec == "fp64" else torch.float32
    cell = fftg.Cell(N, ph, PL, precision=precision, nrhs_tangent=0)
    cell.set_state(np.concatenate([E, np.zeros(6 * N ** 3), ep.ravel(), eb.ravel()]))
    cell.constitutive(eps=_dev(eps, torch.float64))
    st, res = _oracle_state(N, ph, E, eps, ep, eb)
    seq = np.where(res.seq_tr > 0.0, res.seq_tr, 1.0)
    b = np.where(res.plastic, 4 * res.G ** 2 * (res.dgamma / seq - 1.0 / (3 * res.G + res.slope)), 0.0)
    assert (b > 0).mean() > 0.005 and (b < 0).mean() > 0.3
    rng = np.random.default_rng(9)
    p = O.to_comps(O.project(O.to_tensor(rng.standard_normal((6, N, N, N)))))
    if prec == "fp32":
        p = p.astype(np.float32).astype(np.float64)
    q, pq = cell.matvec(_dev(p, dt))
    q = q.double().cpu().numpy().reshape(6, N, N, N)
    qr = O.matvec(O.Tangent(res), O.to_tensor(p))
    ref = O.to_comps(qr)
    cscale = 3.0 * max(1.0, np.abs(O.j2_tangent(res)).max())
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.linalg.norm(q - ref) <= tol * cscale * np.linalg.norm(p)
    cell.close()


def _laminate_table2():
    el = I.Phase(0.833, G, 1e9, 0.0)
    pl = I.Phase(0.833, G, 0.01 * G, 0.05 * G, 0.1)
    N = 15
    return N, I.laminate(N, 5, axis=0), (el, pl)


def test_step_fp64_paper_laminate_matches_oracle():
    N, ph, mats = _laminate_table2()
    dE = np.array([0, 0, 0, 0, 0, 0.05])
    st = O.State(N, ph, mats)
    r = O.solve_increment(st, dE, 1e-6, 1e-12)
    cell = fftg.Cell(N, ph, mats, precision="fp64")
    sig, nn, nc = cell.step(dE, 1e-6, 1e-12)
    assert np.abs(sig - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()
    assert (nn, nc) == (r.newton_iters, r.cg_iters)
    s = cell.stats()
    # quadratic Newton convergence, as in the paper's Table 3
    d = s["newton_norm"]
    assert len(d) >= 3 and d[-1] <= 1e-6
    for a, bb in zip(d[:-1], d[1:]):
        if a > 1e-8:
            assert bb <= 10.0 * a * a
    eps = cell.field(fftg.FFTG_FIELD_STRAIN)
    eps_ref = O.to_comps(st.eps_star) + dE[:, None, None, None]
    assert np.linalg.norm(eps - eps_ref) <= 1e-9 * np.linalg.norm(eps_ref)
    cell.close()


def test_step_mixed_paper_laminate_reaches_fp64():
    N, ph, mats = _laminate_table2()
    dE = np.array([0, 0, 0, 0, 0, 0.05])
    st = O.State(N, ph, mats)
    r = O.solve_increment(st, dE, 1e-6, 1e-12)
    cell = fftg.Cell(N, ph, mats, precision="mixed")
    sig, nn, nc = cell.step(dE, 1e-6, 1e-12)
    assert cell.stats()["newton_norm"][-1] <= 1e-6
    assert np.abs(sig - r.sigma).max() <= 1e-6 * np.abs(r.sigma).max()
    cell.close()


def test_step_fp64_powerlaw_spheres_matches_oracle():
    N = 15
    ph, _, _ = I.random_spheres(N, 0.3, 31, r_min=2.0, r_max=4.0)
    mats = (I.Phase(0.833, G, 0.003, 0.01, 0.3), I.Phase(0.833, G, 0.006, 0.02, 2.0))
    dEs = I.shear_path(0.02, 20)[:4]
    st = O.State(N, ph, mats)
    cell = fftg.Cell(N, ph, mats, precision="fp64")
    for dE in dEs:
        r = O.solve_increment(st, dE, 1e-5, 1e-8)
        sig, nn, nc = cell.step(dE, 1e-5, 1e-8)
        assert np.abs(sig - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()
        assert (nn, nc) == (r.newton_iters, r.cg_iters)
    eb = cell.field(fftg.FFTG_FIELD_EPBAR)
    assert (eb > 0).mean() > 0.1
    assert np.abs(eb - st.epbar).max() <= 1e-10 * np.abs(st.epbar).max()
    cell.close()
