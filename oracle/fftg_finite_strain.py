"""Plain FP64 CPU oracle of the finite-strain extension of the FFT-Galerkin
Newton-CG method.

TEST INFRASTRUCTURE ONLY. Only the tests and the smoke check may import this
module; the product path never calls it and shares no code with it.

The paper states the method for small strains and names finite strain as
the next step (Section 6). The extension here keeps its structure and
replaces the strain by the deformation gradient:

* unknown: F = Fbar + F*, F* a compatible (gradient) fluctuation with zero
  mean, Fbar the prescribed macroscopic deformation gradient;
* equilibrium, as Eq. (linear_system) with the first Piola-Kirchhoff stress:
  G P(F) = 0, where G projects onto gradient fields. In Fourier space a
  gradient field is a (x) xi (row i proportional to xi), and the orthogonal
  projection onto such fields is Ghat : A = (A xi) (x) xi / |xi|^2, i.e.
  Ghat_ijlm = delta_il xi_j xi_m / |xi|^2, with Ghat(0) = 0;
* Newton as Algorithm 1: G K(F) : dF* = -G P(F), K = dP/dF, solved by CG
  with the plain Frobenius product sum_ij A_ij B_ij (F is not symmetric);
  stop on ||dF*|| / (sqrt(V) ||Fbar - I||_F) <= eta_NW after at least one
  iteration;
* material: St. Venant-Kirchhoff per phase (the paper names no finite-strain
  law): E = (F^T F - I)/2, S = lambda tr(E) I + 2 mu E, P = F S, with the
  tangent K_iJkL = delta_ik S_JL + lambda F_iJ F_kL
                   + mu ((F F^T)_ik delta_JL + F_iL F_kJ).

Fields are full tensors [3, 3, N, N, N] (x1 slowest). The DFT convention and
the CG readings (recursive residual, roundoff floor 1e-13 ||P||) are those
of the small-strain oracle.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ROUNDOFF_RHS = 1e-13
I2 = np.eye(3)


def frequencies(N: int) -> np.ndarray:
    """Reduced frequency index of grid index j: j if j <= (N-1)/2, else j - N."""
    k = np.arange(N)
    return np.where(k <= (N - 1) // 2, k, k - N).astype(np.float64)


def ghat_fs(xi):
    """Ghat_ijlm = delta_il xi_j xi_m / |xi|^2 (0 at xi = 0), [3, 3, 3, 3]."""
    xi = np.asarray(xi, dtype=np.float64)
    q2 = float(xi @ xi)
    if q2 == 0.0:
        return np.zeros((3, 3, 3, 3))
    return np.einsum("il,j,m->ijlm", I2, xi, xi) / q2


_GHAT_CACHE = {}


def ghat_fs_field(N: int) -> np.ndarray:
    """Ghat_fs at every frequency of an N^3 grid, [3, 3, 3, 3, N, N, N]
    (frequency index (a, b, c) of axes (x1, x2, x3)). The explicit array
    holds 81 N^3 doubles (cached per N): meant for the small grids of the
    tests (N <= 45 takes 60 MB)."""
    if N not in _GHAT_CACHE:
        k = frequencies(N)
        xi = np.stack(np.meshgrid(k, k, k, indexing="ij"))          # [3, N, N, N]
        q2 = np.sum(xi * xi, axis=0)
        inv = np.where(q2 > 0, 1.0 / np.where(q2 > 0, q2, 1.0), 0.0)
        _GHAT_CACHE[N] = np.einsum("il,j...,m...->ijlm...", I2, xi, xi) * inv
    return _GHAT_CACHE[N]


def project_fs(A):
    """G A for a real field A [3, 3, N, N, N]: forward DFT (numpy FFT scaled
    by 1/|N|), Ghat_fs : A at every frequency (the explicit 3^4 array
    contracted over (l, m)), inverse DFT; the imaginary part must vanish."""
    N = A.shape[-1]
    Ah = np.fft.fftn(A, axes=(2, 3, 4)) / N ** 3
    out = np.einsum("ijlm...,lm...->ij...", ghat_fs_field(N), Ah)
    res = np.fft.ifftn(out, axes=(2, 3, 4)) * N ** 3
    scale = max(np.abs(A).max(), 1e-300)
    assert np.abs(res.imag).max() <= 1e-12 * scale
    return res.real


def inner(A, B) -> float:
    return float(np.sum(A * B))


@dataclass
class SVKResult:
    F: np.ndarray      # [3, 3, ...]
    S: np.ndarray      # second Piola-Kirchhoff stress
    P: np.ndarray      # first Piola-Kirchhoff stress
    lam: np.ndarray
    mu: np.ndarray


def svk_update(F, lam, mu):
    """St. Venant-Kirchhoff: E = (F^T F - I)/2, S = lam tr(E) I + 2 mu E, P = F S."""
    Ib = I2.reshape(3, 3, *([1] * (F.ndim - 2)))
    E = 0.5 * (np.einsum("ki...,kj...->ij...", F, F) - Ib)
    trE = E[0, 0] + E[1, 1] + E[2, 2]
    S = lam * trE * Ib + 2.0 * mu * E
    P = np.einsum("ik...,kj...->ij...", F, S)
    return SVKResult(F, S, P, lam, mu)


def svk_energy(F, lam, mu):
    """W = lam/2 (tr E)^2 + mu E : E."""
    Ib = I2.reshape(3, 3, *([1] * (F.ndim - 2)))
    E = 0.5 * (np.einsum("ki...,kj...->ij...", F, F) - Ib)
    trE = E[0, 0] + E[1, 1] + E[2, 2]
    return 0.5 * lam * trE ** 2 + mu * np.sum(E * E, axis=(0, 1))


def svk_tangent(res: SVKResult, sl=slice(None)):
    """K_iJkL = delta_ik S_JL + lam F_iJ F_kL + mu ((F F^T)_ik delta_JL + F_iL F_kJ),
    [3, 3, 3, 3, M] for the voxels in `sl`."""
    F = res.F.reshape(3, 3, -1)[:, :, sl]
    S = res.S.reshape(3, 3, -1)[:, :, sl]
    lam = np.broadcast_to(res.lam, res.F.shape[2:]).reshape(-1)[sl]
    mu = np.broadcast_to(res.mu, res.F.shape[2:]).reshape(-1)[sl]
    FFt = np.einsum("imv,kmv->ikv", F, F)
    K = np.einsum("ik,JLv->iJkLv", I2, S)
    K += np.einsum("v,iJv,kLv->iJkLv", lam, F, F)
    K += np.einsum("v,ikv,JL->iJkLv", mu, FFt, I2)
    K += np.einsum("v,iLv,kJv->iJkLv", mu, F, F)
    return K


class Tangent:
    CHUNK = 1 << 15

    def __init__(self, res: SVKResult):
        self.res = res
        self.V = int(np.prod(res.F.shape[2:]))

    def apply(self, A):
        Af = A.reshape(3, 3, -1)
        out = np.empty_like(Af)
        for s in range(0, self.V, self.CHUNK):
            sl = slice(s, min(s + self.CHUNK, self.V))
            out[:, :, sl] = np.einsum("ijklv,klv->ijv", svk_tangent(self.res, sl), Af[:, :, sl])
        return out.reshape(A.shape)


def cg(apply_A, b, tol, max_iter=2000, floor=0.0):
    """Hestenes-Stiefel CG with x_0 = 0; stops when ||r|| <= max(tol ||r_0||, floor)."""
    x = np.zeros_like(b)
    r = b.copy()
    rr = inner(r, r)
    rr0 = rr
    if rr0 == 0.0:
        return x, 0
    stop2 = max(tol * tol * rr0, floor * floor)
    p = r.copy()
    it = 0
    while rr > stop2 and it < max_iter:
        q = apply_A(p)
        alpha = rr / inner(p, q)
        x += alpha * p
        r -= alpha * q
        rr_new = inner(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


@dataclass
class State:
    N: int
    phase: np.ndarray
    mats: tuple                 # per phase (lambda, mu)
    Fbar: np.ndarray = field(default=None)
    Fstar: np.ndarray = field(default=None)

    def __post_init__(self):
        tab = np.array([tuple(m) for m in self.mats], dtype=np.float64)
        ph = np.asarray(self.phase).astype(np.int64)
        self.lam, self.mu = tab[ph, 0], tab[ph, 1]
        if self.Fbar is None:
            self.Fbar = np.eye(3)
        if self.Fstar is None:
            self.Fstar = np.zeros((3, 3) + (self.N,) * 3)

    def material(self, Fbar, Fstar):
        return svk_update(Fstar + Fbar[:, :, None, None, None], self.lam, self.mu)


@dataclass
class StepResult:
    P: np.ndarray               # homogenised first Piola-Kirchhoff stress [3, 3]
    newton_iters: int
    cg_iters: int
    newton_norms: list
    cg_per_newton: list
    residual: list             # ||G P|| / ||P|| before each solve
    converged: bool


def solve_increment(st: State, dFbar, tol_newton, tol_cg, max_newton=50, max_cg=2000):
    """One increment (Algorithm 1 with F in place of the strain): Fbar +=
    dFbar, Newton on G P(Fbar + F*) = 0 from the previous F*, each iteration
    solving G K dF* = -G P by CG. dFbar is a 3x3 matrix (or 9 numbers, row
    major). Updates `st` when Newton converges."""
    Fbar = st.Fbar + np.asarray(dFbar, dtype=np.float64).reshape(3, 3)
    Fs = st.Fstar.copy()
    V = st.N ** 3
    normH = np.sqrt(V * np.sum((Fbar - I2) ** 2))
    it = cgt = 0
    norms, cgs, resid = [], [], []
    converged = False
    while True:
        res = st.material(Fbar, Fs)
        GP = project_fs(res.P)
        nG, nP = np.sqrt(inner(GP, GP)), np.sqrt(inner(res.P, res.P))
        resid.append(nG / nP if nP > 0 else 0.0)
        tan = Tangent(res)
        if nG <= ROUNDOFF_RHS * nP:
            dF, ncg = np.zeros_like(GP), 0
        else:
            dF, ncg = cg(lambda p: project_fs(tan.apply(p)), -GP, tol_cg, max_cg,
                         floor=ROUNDOFF_RHS * nP)
        Fs += dF
        it += 1
        cgt += ncg
        cgs.append(ncg)
        nd = np.sqrt(inner(dF, dF))
        rel = nd / normH if normH > 0 else (0.0 if nd == 0 else np.inf)
        norms.append(rel)
        if rel <= tol_newton or nd == 0.0:
            converged = True
            break
        if it >= max_newton:
            break
    res = st.material(Fbar, Fs)
    Pbar = res.P.reshape(3, 3, -1).mean(axis=-1)
    if converged:
        st.Fbar = Fbar
        st.Fstar = Fs
    return StepResult(Pbar, it, cgt, norms, cgs, resid, converged)


def macro_tangent(st: State, tol_cg, max_cg=2000):
    """9x9 macroscopic tangent dPbar/dFbar at the committed state (row major
    pairs: C[3i+j, 3k+l] = dPbar_ij / dFbar_kl): for each unit tensor E_kl,
    CG on G K x = -G (K : E_kl) (the linearised equilibrium with the
    macroscopic perturbation), then column (kl) = mean(K : (E_kl + x)).
    Returns (C, CG iterations summed over the nine solves)."""
    res = st.material(st.Fbar, st.Fstar)
    tan = Tangent(res)
    shape = (3, 3) + (st.N,) * 3
    C = np.zeros((9, 9))
    total = 0
    for col in range(9):
        E = np.zeros(shape)
        E[col // 3, col % 3] = 1.0
        KE = tan.apply(E)
        rhs = -project_fs(KE)
        nKE = np.sqrt(inner(KE, KE))
        if np.sqrt(inner(rhs, rhs)) <= ROUNDOFF_RHS * nKE:
            x, n = np.zeros(shape), 0
        else:
            x, n = cg(lambda p: project_fs(tan.apply(p)), rhs, tol_cg, max_cg,
                      floor=ROUNDOFF_RHS * nKE)
        total += n
        C[:, col] = tan.apply(E + x).reshape(9, -1).mean(axis=-1)
    return C, total
