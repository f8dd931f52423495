"""Plain FP64 CPU oracle of the FFT-Galerkin Newton-CG method.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module; the product path never
calls it and shares no code with it.

Everything is written in full 3x3 tensor notation, in float64, vectorised
over voxels but otherwise in the order the paper states it:

* grid and frequencies ............ Section 2.3 (reduced index set, odd N)
* DFT pair F, F^-1 ................ Eq. (DFT_forward_inverse); numpy's FFT is
                                    the library primitive, scaled to the
                                    paper's convention (1/|N| on the forward);
                                    a textbook mixed-radix Cooley-Tukey FFT
                                    (`fft_textbook`) written from the DFT sum
                                    can replace it (FFT_IMPL = "textbook") and
                                    pins it beyond the sizes a dense DFT
                                    reaches
* projection G = F^-1 Ghat F ...... Eq. (discrete_projection), Ghat from the
                                    closed form of Appendix A, Eq. (FT_projection)
* reference-medium Green operator . Appendix A, Eq. (Gamma_explicit), used only
                                    to pin Ghat by an independent formula
* J2 return mapping and tangent ... Section 4.2 (hardening sigma_0 + H epbar^n;
                                    closed-form return for n = 1, a bracketed
                                    scalar Newton for other n)
* CG on G C de = -G sigma ......... Eq. (linear_system), Section 2.5
* Newton increment loop ........... Algorithm 1
* homogenised stress .............. Eq. (trapz): the mean of the nodal stress
* macroscopic 6x6 tangent ......... not in the paper (FE^2 context of
                                    Section 1); six linear solves with the
                                    converged tangent

Readings of the paper taken here (each also listed in the design notes):
* plastic iff Phi_trial > 1e-12 * sigma_0 (tie-break at the yield surface);
* Newton stops on ||de*|| / ||E||_field <= eta_NW with the field L2 norm and
  ||E||_field = sqrt(V) ||E||_F, after at least one iteration;
* CG stops on the recursive residual ||r_j|| / ||r_0|| <= eta_CG, x_0 = 0;
  a right-hand side at roundoff level, ||G sigma|| <= 1e-13 ||sigma||, is
  already in equilibrium and takes no CG iteration (de = 0), and CG also
  stops once ||r_j|| <= 1e-13 ||tau||, tau the field whose projection is the
  right-hand side (sigma, or C : E_j for the macroscopic tangent): below that
  floor the residual is FFT roundoff, which has an incompatible part that CG
  cannot remove, and iterating on it makes the iterate diverge;
* the history is committed from one last constitutive call at the converged
  strain, and the converged eps* is the initial guess of the next increment.

Field layout: full tensors [3, 3, N, N, N] (x1 slowest). The 6-component
order used at the library boundary is (11, 22, 33, 23, 13, 12).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))

# A residual below this fraction of the norm of the field it was projected
# from is FFT roundoff (see the readings above).
ROUNDOFF_RHS = 1e-13

I2 = np.eye(3)
II = np.einsum("ij,lm->ijlm", I2, I2)
I4s = 0.5 * (np.einsum("il,jm->ijlm", I2, I2) + np.einsum("im,jl->ijlm", I2, I2))
I4d = I4s - II / 3.0


# --------------------------------------------------------------------------
# 6-component <-> full tensor conversion (boundary convention only)
# --------------------------------------------------------------------------
def to_tensor(v6):
    """[6, ...] tensor components (11,22,33,23,13,12) -> [3, 3, ...]."""
    v6 = np.asarray(v6, dtype=np.float64)
    t = np.zeros((3, 3) + v6.shape[1:])
    for c, (i, j) in enumerate(PAIRS):
        t[i, j] = v6[c]
        t[j, i] = v6[c]
    return t


def to_comps(t):
    """[3, 3, ...] symmetric tensor -> [6, ...] components."""
    return np.stack([t[i, j] for (i, j) in PAIRS])


# --------------------------------------------------------------------------
# Grid, frequencies and the DFT pair (Section 2.3)
# --------------------------------------------------------------------------
def frequencies(N: int) -> np.ndarray:
    """Index j in [0, N) -> frequency k in the reduced set -N/2 < k < N/2."""
    j = np.arange(N)
    return np.where(j <= (N - 1) // 2, j, j - N)


# Which FFT evaluates the DFT sums: "library" (numpy's pocketfft, the
# default: about ten times faster, which the full-size parity tests need) or
# "textbook" (`fft_textbook` below). Both compute the same sums.
FFT_IMPL = "library"


def _smallest_factor(n: int) -> int:
    f = 2
    while f * f <= n:
        if n % f == 0:
            return f
        f += 1
    return n


def _cooley_tukey(x, sign):
    """DFT X[k] = sum_n x[n] exp(sign 2 pi i n k / N) along the last axis,
    N = x.shape[-1], by recursive decimation in time over the smallest prime
    factor p of N (N = p m):

      n = j + p n1 (j < p, n1 < m), k = k1 + m k2 (k1 < m, k2 < p):
      X[k1 + m k2] = sum_j w_p^(j k2) [w_N^(j k1) Y_j[k1]],
      Y_j = the m-point DFT of the subsequence x[j + p n1],

    w_L = exp(sign 2 pi i / L); a prime length is summed directly."""
    N = x.shape[-1]
    if N == 1:
        return x.copy()
    p = _smallest_factor(N)
    if p == N:
        n = np.arange(N)
        W = np.exp(sign * 2j * np.pi * np.outer(n, n) / N)
        return x @ W.T
    m = N // p
    # [..., j, n1] = x[j + p n1]
    sub = np.swapaxes(x.reshape(x.shape[:-1] + (m, p)), -1, -2)
    Y = _cooley_tukey(np.ascontiguousarray(sub), sign)
    j = np.arange(p)
    Y = Y * np.exp(sign * 2j * np.pi * np.outer(j, np.arange(m)) / N)
    Wp = np.exp(sign * 2j * np.pi * np.outer(j, j) / p)
    X = np.empty_like(Y)
    for k2 in range(p):
        acc = Y[..., 0, :].copy()
        for jj in range(1, p):
            acc += Wp[k2, jj] * Y[..., jj, :]
        X[..., k2, :] = acc
    return X.reshape(x.shape)


def fft_textbook(x, axes=(-3, -2, -1), sign=-1):
    """Unscaled multi-dimensional DFT, sum_n x[n] exp(sign 2 pi i n.k / N)
    over `axes`, one axis at a time with the mixed-radix Cooley-Tukey
    recursion above (radices 3 and 5 for the grids of this method)."""
    x = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        y = np.ascontiguousarray(np.moveaxis(x, ax, -1))
        x = np.moveaxis(_cooley_tukey(y, sign), -1, ax)
    return x


def dft_forward(t):
    """F: Fourier coefficients with the 1/|N| factor on the forward sum."""
    N3 = np.prod(t.shape[-3:])
    if FFT_IMPL == "textbook":
        return fft_textbook(t, sign=-1) / N3
    return np.fft.fftn(t, axes=(-3, -2, -1)) / N3


def dft_inverse(th):
    """F^-1: nodal values, no factor on the inverse sum."""
    N3 = np.prod(th.shape[-3:])
    if FFT_IMPL == "textbook":
        return fft_textbook(th, sign=+1)
    return np.fft.ifftn(th, axes=(-3, -2, -1)) * N3


def dft_forward_dense(t):
    """Brute-force dense DFT of Eq. (DFT_forward_inverse)_1 (tiny grids only).

    Entry [k, m] of each 1D matrix is exp(-2 pi i k m / N) with k the reduced
    frequency stored at index j (k = j or j - N) and m the node index; the 3D
    matrix is their Kronecker product. Used to pin `dft_forward`.
    """
    N1, N2, N3 = t.shape[-3:]
    mats = []
    for n in (N1, N2, N3):
        k = frequencies(n)
        m = np.arange(n)
        mats.append(np.exp(-2j * np.pi * np.outer(k, m) / n))
    M = np.kron(np.kron(mats[0], mats[1]), mats[2])
    flat = t.reshape(t.shape[:-3] + (N1 * N2 * N3,))
    out = flat @ M.T / (N1 * N2 * N3)
    return out.reshape(t.shape[:-3] + (N1, N2, N3))


# --------------------------------------------------------------------------
# Projection operator (Appendix A)
# --------------------------------------------------------------------------
def ghat(xi):
    """Ghat_ijlm(xi) of Eq. (FT_projection); xi [..., 3]; Ghat(0) = 0."""
    xi = np.asarray(xi, dtype=np.float64)
    n2 = np.sum(xi * xi, axis=-1)
    zero = n2 == 0.0
    n2s = np.where(zero, 1.0, n2)
    d = I2
    t = (np.einsum("...i,jl,...m->...ijlm", xi, d, xi)
         + np.einsum("...i,jm,...l->...ijlm", xi, d, xi)
         + np.einsum("...j,il,...m->...ijlm", xi, d, xi)
         + np.einsum("...j,im,...l->...ijlm", xi, d, xi))
    g = 0.5 * t / n2s[..., None, None, None, None]
    g -= (np.einsum("...i,...j,...l,...m->...ijlm", xi, xi, xi, xi)
          / (n2s ** 2)[..., None, None, None, None])
    g[zero] = 0.0
    return g


def gamma_ref(xi, Cref):
    """Gamma^ref_ijlm(xi) of Eq. (Gamma_explicit) via the acoustic tensor.

    A_il = C_ijlm xi_j xi_m; Gamma = 1/4 (A^-1_jm xi_i xi_l + A^-1_jl xi_i xi_m
    + A^-1_im xi_j xi_l + A^-1_il xi_j xi_m); Gamma(0) = 0.
    """
    xi = np.asarray(xi, dtype=np.float64)
    n2 = np.sum(xi * xi, axis=-1)
    zero = n2 == 0.0
    xs = np.where(zero[..., None], 1.0, xi)
    A = np.einsum("ijlm,...j,...m->...il", Cref, xs, xs)
    Ai = np.linalg.inv(A)
    g = 0.25 * (np.einsum("...jm,...i,...l->...ijlm", Ai, xs, xs)
                + np.einsum("...jl,...i,...m->...ijlm", Ai, xs, xs)
                + np.einsum("...im,...j,...l->...ijlm", Ai, xs, xs)
                + np.einsum("...il,...j,...m->...ijlm", Ai, xs, xs))
    g[zero] = 0.0
    return g


def project(tau):
    """G tau = F^-1 [Ghat : F[tau]] for a real field tau [3, 3, N, N, N].

    Eq. (discrete_projection). Ghat is evaluated one k1-slice at a time so
    that large grids fit in memory; no other reordering. The imaginary part
    left by the inverse transform must vanish (G is a real matrix); it is
    checked and dropped.
    """
    N1, N2, N3 = tau.shape[-3:]
    th = dft_forward(tau)
    out = np.empty_like(th)
    k2 = frequencies(N2)
    k3 = frequencies(N3)
    for a, k1 in enumerate(frequencies(N1)):
        xi = np.stack(np.broadcast_arrays(np.float64(k1), k2[:, None] * 1.0,
                                          k3[None, :] * 1.0), axis=-1)
        g = ghat(xi)  # [N2, N3, 3, 3, 3, 3]
        out[:, :, a] = np.einsum("bcijlm,lmbc->ijbc", g, th[:, :, a])
    res = dft_inverse(out)
    scale = max(np.abs(tau).max(), 1e-300)
    assert np.abs(res.imag).max() <= 1e-12 * scale, "G tau not real"
    return res.real


def inner(a, b) -> float:
    """Double contraction summed over nodes, Eq. (trapz) without the weight."""
    return float(np.sum(a * b))


# --------------------------------------------------------------------------
# J2 elasto-plasticity with isotropic hardening sigma_0 + H epbar^n (Section 4.2)
# --------------------------------------------------------------------------
@dataclass
class J2Result:
    sigma: np.ndarray        # [3, 3, ...]
    eps_p: np.ndarray        # [3, 3, ...] trial (updated) plastic strain
    epbar: np.ndarray        # [...] trial accumulated plastic strain
    plastic: np.ndarray      # [...] bool
    dgamma: np.ndarray       # [...]
    seq_tr: np.ndarray       # [...] trial von Mises stress
    Ntr: np.ndarray          # [3, 3, ...] trial flow direction
    K: np.ndarray
    G: np.ndarray
    H: np.ndarray
    slope: np.ndarray        # [...] n H (epbar_t + dgamma)^(n-1): hardening slope
                             # at the returned state (H for n = 1)


MODEL_J2, MODEL_NLELASTIC, MODEL_VISCO = 0, 1, 2


@dataclass
class MatFields:
    """Per-voxel material parameters (Section 4): bulk and shear moduli,
    sigma_0, H, exponent n, eps_0, t_0 and the model id."""
    K: np.ndarray
    G: np.ndarray
    sy: np.ndarray
    H: np.ndarray
    n: np.ndarray
    eps0: np.ndarray
    t0: np.ndarray
    model: np.ndarray


def material_fields(phase, mats):
    """Per-voxel parameters from a phase map. A material is an object with
    as_tuple() or a tuple (K, G, sigma_y, H[, n]) (J2, n = 1 by default) or
    (K, G, sigma_0, H, n, eps_0, t_0, model)."""
    rows = []
    for m in mats:
        t = tuple(float(v) for v in (m.as_tuple() if hasattr(m, "as_tuple") else m))
        if len(t) == 4:
            t = t + (1.0,)
        if len(t) == 5:
            t = t + (0.0, 0.0, float(MODEL_J2))
        rows.append(t)
    tab = np.array(rows, dtype=np.float64)
    ph = np.asarray(phase).astype(np.int64)
    return MatFields(*(tab[ph, j] for j in range(7)), tab[ph, 7].astype(np.int64))


def power_law_dgamma(seq_tr, epbar_t, G, sy, H, n, max_iter=200):
    """Root dgamma > 0 of the scalar return equation of Section 4.2,
        seq_tr - 3 G dgamma - sigma_0 - H (epbar_t + dgamma)^n = 0,
    for trial states with Phi_tr > 0 (arrays of equal shape).

    The left side is positive at 0 and non-positive at Phi_tr / (3G) (the
    hardening term only grows), so the root is bracketed there; Newton steps
    that leave the current bracket are replaced by bisection. Iterates until
    the bracket or the step is at the last few bits.
    """
    seq_tr, epbar_t, G, sy, H, n = np.broadcast_arrays(
        *(np.asarray(v, dtype=np.float64) for v in (seq_tr, epbar_t, G, sy, H, n)))
    phi_tr = seq_tr - (sy + H * epbar_t ** n)
    lo = np.zeros_like(seq_tr)
    hi = phi_tr / (3.0 * G)
    x = 0.5 * (lo + hi)
    for _ in range(max_iter):
        y = epbar_t + x
        f = seq_tr - 3.0 * G * x - sy - H * y ** n
        lo = np.where(f > 0.0, x, lo)
        hi = np.where(f > 0.0, hi, x)
        with np.errstate(divide="ignore", invalid="ignore"):
            df = -3.0 * G - n * H * np.where(y > 0.0, y ** (n - 1.0), np.inf)
            xn = x - f / df
        bad = ~((xn > lo) & (xn < hi)) | ~np.isfinite(xn)
        xn = np.where(bad, 0.5 * (lo + hi), xn)
        done = np.abs(xn - x) <= 4.0 * np.finfo(float).eps * np.maximum(np.abs(x), 1e-300)
        x = xn
        if np.all(done | (hi - lo <= 4.0 * np.finfo(float).eps * hi)):
            break
    return x


def j2_update(eps, eps_p_t, epbar_t, K, G, sy, H, n=None, tie=1e-12):
    """Backward-Euler elastic predictor / plastic corrector.

    eps, eps_p_t: [3, 3, ...]; epbar_t, K, G, sy, H, n: [...] (n = None:
    linear hardening, n = 1). Trial state (Eq. model:plas:trial), elastic
    branch (Eq. model:plas:elas), plastic corrector (Eq. model:plas:corrector)
    with dgamma from the scalar return equation: in closed form,
    Phi_tr / (3G + H), for n = 1 and by `power_law_dgamma` otherwise.
    """
    if n is None:
        n = np.ones_like(np.asarray(epbar_t, dtype=np.float64))
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), np.shape(epbar_t))
    ee = eps - eps_p_t
    tr = ee[0, 0] + ee[1, 1] + ee[2, 2]
    dev = ee - tr / 3.0 * I2.reshape(3, 3, *([1] * (ee.ndim - 2)))
    sig_tr = K * tr * I2.reshape(3, 3, *([1] * (ee.ndim - 2))) + 2.0 * G * dev
    s = sig_tr - (sig_tr[0, 0] + sig_tr[1, 1] + sig_tr[2, 2]) / 3.0 * \
        I2.reshape(3, 3, *([1] * (ee.ndim - 2)))
    seq = np.sqrt(1.5 * np.sum(s * s, axis=(0, 1)))
    phi = seq - (sy + H * epbar_t ** n)
    plastic = phi > tie * sy
    seq_safe = np.where(seq > 0.0, seq, 1.0)
    Ntr = 1.5 * s / seq_safe
    linear = n == 1.0
    dgamma = np.where(plastic & linear, phi / (3.0 * G + H), 0.0)
    pw = plastic & ~linear
    if np.any(pw):
        b = np.broadcast_arrays(seq, epbar_t, G, sy, H, n)
        dgamma = dgamma.copy()
        dgamma[pw] = power_law_dgamma(*(v[pw] for v in b))
    with np.errstate(divide="ignore", invalid="ignore"):
        y = epbar_t + dgamma
        slope = np.where(linear, H, n * H * np.where(y > 0.0, y ** (n - 1.0), 0.0))
    eps_p = eps_p_t + dgamma * Ntr
    epbar = epbar_t + dgamma
    ee2 = eps - eps_p
    tr2 = ee2[0, 0] + ee2[1, 1] + ee2[2, 2]
    dev2 = ee2 - tr2 / 3.0 * I2.reshape(3, 3, *([1] * (ee.ndim - 2)))
    sigma = K * tr2 * I2.reshape(3, 3, *([1] * (ee.ndim - 2))) + 2.0 * G * dev2
    return J2Result(sigma, eps_p, epbar, plastic, dgamma, seq, Ntr, K, G, H,
                    np.broadcast_to(slope, np.shape(epbar_t)))


def j2_tangent(res: J2Result, sl=slice(None)):
    """Consistent tangent C_ijlm, [3, 3, 3, 3, M] for the voxels in `sl`.

    Elastic: C = C_e = K I(x)I + 2G I_d. Plastic (Section 4.2):
    C = C_e - 6 G^2 dgamma / seq_tr I_d
            + 4 G^2 (dgamma / seq_tr - 1/(3G + n H (epbar_t + dgamma)^(n-1))) N(x)N.
    """
    K = res.K.reshape(-1)[sl]
    G = res.G.reshape(-1)[sl]
    hs = res.slope.reshape(-1)[sl]
    dg = res.dgamma.reshape(-1)[sl]
    seq = res.seq_tr.reshape(-1)[sl]
    pl = res.plastic.reshape(-1)[sl]
    Nt = res.Ntr.reshape(3, 3, -1)[:, :, sl]
    C = (np.einsum("ijlm,v->ijlmv", II, K)
         + np.einsum("ijlm,v->ijlmv", I4d, 2.0 * G))
    seqs = np.where(seq > 0.0, seq, 1.0)
    a = np.where(pl, 6.0 * G * G * dg / seqs, 0.0)
    b = np.where(pl, 4.0 * G * G * (dg / seqs - 1.0 / (3.0 * G + hs)), 0.0)
    C -= np.einsum("ijlm,v->ijlmv", I4d, a)
    C += np.einsum("ijv,lmv,v->ijlmv", Nt, Nt, b)
    return C


# --------------------------------------------------------------------------
# Non-linear elasticity (Section 4.1)
# --------------------------------------------------------------------------
@dataclass
class NLEResult:
    sigma: np.ndarray        # [3, 3, ...]
    eps_p: np.ndarray        # history, unchanged (the model has none)
    epbar: np.ndarray
    K: np.ndarray
    s0: np.ndarray
    e0: np.ndarray
    n: np.ndarray
    eeq: np.ndarray          # [...] equivalent strain
    Nd: np.ndarray           # [3, 3, ...] N = 2/3 eps_d / eps_eq (0 where eps_eq = 0)


def nonlinear_elastic_update(eps, eps_p_t, epbar_t, K, s0, e0, n):
    """sigma = K tr(eps) I + sigma_0 (eps_eq / eps_0)^n N with
    N = 2/3 eps_d / eps_eq and eps_eq = sqrt(2/3 eps_d : eps_d)
    (Eqs. model:nlin:stress, model:nlin:N); no history."""
    Ib = I2.reshape(3, 3, *([1] * (eps.ndim - 2)))
    tr = eps[0, 0] + eps[1, 1] + eps[2, 2]
    ed = eps - tr / 3.0 * Ib
    eeq = np.sqrt(2.0 / 3.0 * np.sum(ed * ed, axis=(0, 1)))
    safe = np.where(eeq > 0.0, eeq, 1.0)
    Nd = np.where(eeq > 0.0, 2.0 / 3.0 * ed / safe, 0.0)
    sigma = K * tr * Ib + s0 * (eeq / e0) ** n * Nd
    return NLEResult(sigma, eps_p_t.copy(), np.array(epbar_t, dtype=np.float64, copy=True),
                     K, s0, e0, n, eeq, Nd)


def nle_tangent(res: NLEResult, sl=slice(None)):
    """C = K I(x)I + sigma_0/eps_eq (eps_eq/eps_0)^n ((n - 1) N(x)N + 2/3 I_d)
    (Eq. model:nlin-tangent). At eps_eq = 0 the factor sigma_0/eps_eq
    (eps_eq/eps_0)^n is taken as its limit sigma_0/eps_0 for n = 1 and as 0
    otherwise."""
    K = res.K.reshape(-1)[sl]
    s0 = res.s0.reshape(-1)[sl]
    e0 = res.e0.reshape(-1)[sl]
    n = res.n.reshape(-1)[sl]
    eeq = res.eeq.reshape(-1)[sl]
    Nd = res.Nd.reshape(3, 3, -1)[:, :, sl]
    safe = np.where(eeq > 0.0, eeq, 1.0)
    c = np.where(eeq > 0.0, s0 / safe * (eeq / e0) ** n, np.where(n == 1.0, s0 / e0, 0.0))
    C = np.einsum("ijlm,v->ijlmv", II, K)
    C += np.einsum("ijlm,v->ijlmv", I4d, 2.0 / 3.0 * c)
    C += np.einsum("ijv,lmv,v->ijlmv", Nd, Nd, c * (n - 1.0))
    return C


# --------------------------------------------------------------------------
# Visco-plasticity (Section 4.3)
# --------------------------------------------------------------------------
def visco_dgamma(seq_tr, G, s0, gdt, n, max_iter=200):
    """Root of the implicit backward-Euler equation of Section 4.3,
        dgamma = gamma_0 dt ((seq_tr - 3 G dgamma) / sigma_0)^(1/n),
    gamma_0 = eps_0 / t_0, for seq_tr > 0: g(x) = x - gamma_0 dt ((seq_tr -
    3 G x) / sigma_0)^(1/n) is increasing, negative at 0 and positive at
    seq_tr / (3G); Newton steps leaving the bracket become bisections."""
    seq_tr, G, s0, gdt, n = np.broadcast_arrays(
        *(np.asarray(v, dtype=np.float64) for v in (seq_tr, G, s0, gdt, n)))
    lo = np.zeros_like(seq_tr)
    hi = seq_tr / (3.0 * G)
    x = 0.5 * hi
    for _ in range(max_iter):
        u = np.maximum(seq_tr - 3.0 * G * x, 0.0) / s0
        g = x - gdt * u ** (1.0 / n)
        lo = np.where(g < 0.0, x, lo)
        hi = np.where(g < 0.0, hi, x)
        with np.errstate(divide="ignore", invalid="ignore"):
            dg = 1.0 + gdt / n * np.where(u > 0.0, u ** (1.0 / n - 1.0), np.inf) * 3.0 * G / s0
            xn = x - g / dg
        bad = ~((xn > lo) & (xn < hi)) | ~np.isfinite(xn)
        xn = np.where(bad, 0.5 * (lo + hi), xn)
        done = np.abs(xn - x) <= 4.0 * np.finfo(float).eps * np.maximum(np.abs(x), 1e-300)
        x = xn
        if np.all(done | (hi - lo <= 4.0 * np.finfo(float).eps * hi)):
            break
    return x


def visco_update(eps, eps_p_t, epbar_t, K, G, s0, e0, t0, n, dt, tie=1e-12):
    """Backward-Euler update of Section 4.3: the elastic trial state of
    Section 4.2, then dgamma from `visco_dgamma` wherever seq_tr > tie
    sigma_0 (there is no elastic range), and the corrector of Eq.
    (model:plas:corrector). The consistent tangent has the form of the J2 one
    with the slope n sigma_0 / (gamma_0 dt) (dgamma / (gamma_0 dt))^(n-1) in
    place of the hardening slope, so the result is returned as a J2Result
    whose `slope` holds it (`H` is unused)."""
    Ib = I2.reshape(3, 3, *([1] * (eps.ndim - 2)))
    ee = eps - eps_p_t
    tr = ee[0, 0] + ee[1, 1] + ee[2, 2]
    s = 2.0 * G * (ee - tr / 3.0 * Ib)
    seq = np.sqrt(1.5 * np.sum(s * s, axis=(0, 1)))
    flow = seq > tie * s0
    safe = np.where(seq > 0.0, seq, 1.0)
    Ntr = 1.5 * s / safe
    gdt = e0 / t0 * dt
    dgamma = np.zeros_like(seq)
    if np.any(flow):
        b = np.broadcast_arrays(seq, G, s0, gdt, n)
        dgamma[flow] = visco_dgamma(*(v[flow] for v in b))
    with np.errstate(divide="ignore", invalid="ignore"):
        q = dgamma / gdt
        slope = np.where(flow, n * s0 / gdt * np.where(q > 0.0, q ** (n - 1.0), 0.0), 0.0)
    eps_p = eps_p_t + dgamma * Ntr
    epbar = epbar_t + dgamma
    ee2 = eps - eps_p
    tr2 = ee2[0, 0] + ee2[1, 1] + ee2[2, 2]
    sigma = K * tr2 * Ib + 2.0 * G * (ee2 - tr2 / 3.0 * Ib)
    return J2Result(sigma, eps_p, epbar, flow, dgamma, seq, Ntr, K, G,
                    np.zeros_like(seq), slope)


@dataclass
class PointResult:
    """Material update of a cell with several models: the fields, and per
    model the voxels (flat indices) and that model's result on them."""
    sigma: np.ndarray
    eps_p: np.ndarray
    epbar: np.ndarray
    parts: list


def point_tangent(res, sl=slice(None)):
    """Consistent tangent [3, 3, 3, 3, M] of the voxels in `sl` (a slice of
    the flat voxel index) for any of the results above."""
    if isinstance(res, J2Result):
        return j2_tangent(res, sl)
    if isinstance(res, NLEResult):
        return nle_tangent(res, sl)
    V = res.epbar.size
    idx = np.arange(V)[sl]
    C = np.zeros((3, 3, 3, 3, idx.size))
    pos = np.full(V, -1)
    pos[idx] = np.arange(idx.size)
    for vox, r in res.parts:
        here = pos[vox] >= 0
        if np.any(here):
            C[..., pos[vox[here]]] = point_tangent(r, np.flatnonzero(here))
    return C


class Tangent:
    """The block-diagonal tangent D of Eq. (local_tangent), applied chunk-wise."""

    CHUNK = 1 << 16

    def __init__(self, res):
        self.res = res
        self.shape = res.sigma.shape[2:]
        self.V = int(np.prod(self.shape))

    def apply(self, p):
        """C : p for a field p [3, 3, N, N, N]."""
        pf = p.reshape(3, 3, -1)
        out = np.empty_like(pf)
        for s in range(0, self.V, self.CHUNK):
            sl = slice(s, min(s + self.CHUNK, self.V))
            C = point_tangent(self.res, sl)
            out[:, :, sl] = np.einsum("ijlmv,lmv->ijv", C, pf[:, :, sl])
        return out.reshape(p.shape)


# --------------------------------------------------------------------------
# Linear solve (Eq. linear_system) by conjugate gradients
# --------------------------------------------------------------------------
def matvec(tangent: Tangent, p):
    """G (C : p) for a compatible field p."""
    return project(tangent.apply(p))


def cg(apply_A, b, tol, max_iter=2000, fixed_iters=None, floor=0.0):
    """Hestenes-Stiefel CG with x_0 = 0 on A x = b, A = G C on E_N.

    Stops when ||r_j|| <= max(tol ||r_0||, floor) (recursive residual) or,
    if fixed_iters is given, after exactly that many iterations.
    Returns (x, iterations, final relative residual).
    """
    x = np.zeros_like(b)
    r = b.copy()
    rr = inner(r, r)
    rr0 = rr
    if rr0 == 0.0:
        return x, 0, 0.0
    stop2 = max(tol * tol * rr0, floor * floor)
    p = r.copy()
    it = 0
    while True:
        if fixed_iters is None:
            if rr <= stop2 or it >= max_iter:
                break
        elif it >= fixed_iters:
            break
        q = apply_A(p)
        alpha = rr / inner(p, q)
        x += alpha * p
        r -= alpha * q
        rr_new = inner(r, r)
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p
        it += 1
    return x, it, float(np.sqrt(rr / rr0))


# --------------------------------------------------------------------------
# The basic scheme (Section 3.2): Richardson's iteration with a reference
# medium, as a comparison solver for the same linear system
# --------------------------------------------------------------------------
def mandel(C):
    """6x6 matrices [6, 6, M] of tangents C [3, 3, 3, 3, M] in the Mandel
    basis (shear components scaled by sqrt 2), whose eigenvalues are those
    of C acting on symmetric tensors with the Frobenius product."""
    w = np.array([1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)])
    M = np.empty((6, 6, C.shape[-1]))
    for a, (i, j) in enumerate(PAIRS):
        for b, (l, m) in enumerate(PAIRS):
            M[a, b] = w[a] * w[b] * C[i, j, l, m]
    return M


def tangent_bounds(res):
    """lambda_min and lambda_max of the local tangents over the grid
    (Section 3.2), from the eigenvalues of each voxel's 6x6 matrix."""
    V = res.epbar.size
    lo, hi = np.inf, -np.inf
    for s0 in range(0, V, Tangent.CHUNK):
        M = mandel(point_tangent(res, slice(s0, min(s0 + Tangent.CHUNK, V))))
        ev = np.linalg.eigvalsh(np.moveaxis(M, -1, 0))
        lo, hi = min(lo, ev.min()), max(hi, ev.max())
    return float(lo), float(hi)


def richardson(apply_A, b, omega, tol, max_iter=2000, floor=0.0):
    """Richardson's iteration x_{k+1} = x_k + omega (b - A x_k), x_0 = 0.

    With the reference medium C_ref = c I_s, c = (lambda_min + lambda_max)/2,
    Gamma_ref = G / c (Appendix A) and the basic scheme's update
    x + Gamma_ref (-sigma - D x) is this iteration on G D x = -G sigma with
    omega = 1 / c. Stops when ||b - A x_k|| <= max(tol ||b||, floor).
    Returns (x, iterations, final relative residual).
    """
    x = np.zeros_like(b)
    r = b.copy()
    rr0 = inner(r, r)
    if rr0 == 0.0:
        return x, 0, 0.0
    stop2 = max(tol * tol * rr0, floor * floor)
    rr = rr0
    it = 0
    while rr > stop2 and it < max_iter:
        x += omega * r
        r = b - apply_A(x)
        rr = inner(r, r)
        it += 1
    return x, it, float(np.sqrt(rr / rr0))


def linear_solve(solver, tan, res, rhs, tol, max_iter, floor, fixed_iters=None):
    """G C x = rhs by CG (solver 'cg') or by the basic scheme ('richardson')."""
    if solver == "cg":
        return cg(lambda p: matvec(tan, p), rhs, tol, max_iter, fixed_iters=fixed_iters, floor=floor)
    lo, hi = tangent_bounds(res)
    return richardson(lambda p: matvec(tan, p), rhs, 2.0 / (lo + hi), tol, max_iter, floor=floor)


# --------------------------------------------------------------------------
# Algorithm 1: incremental-iterative Newton-CG
# --------------------------------------------------------------------------
@dataclass
class State:
    N: int
    phase: np.ndarray
    mats: tuple
    E: np.ndarray = field(default=None)          # [3, 3]
    eps_star: np.ndarray = field(default=None)   # [3, 3, N, N, N]
    eps_p: np.ndarray = field(default=None)      # committed history
    epbar: np.ndarray = field(default=None)
    dt: float = 1.0                              # time step of an increment
                                                 # (rate-dependent models)

    def __post_init__(self):
        N = self.N
        self.mat = material_fields(self.phase, self.mats)
        self.K, self.G, self.sy, self.H, self.n = (self.mat.K, self.mat.G, self.mat.sy,
                                                   self.mat.H, self.mat.n)
        if self.E is None:
            self.E = np.zeros((3, 3))
        if self.eps_star is None:
            self.eps_star = np.zeros((3, 3, N, N, N))
        if self.eps_p is None:
            self.eps_p = np.zeros((3, 3, N, N, N))
        if self.epbar is None:
            self.epbar = np.zeros((N, N, N))

    def constitutive(self, E, eps_star):
        """The material update of Section 4 at E + eps*, voxel by voxel with
        each voxel's model, against the committed history."""
        eps = eps_star + E[:, :, None, None, None]
        mt = self.mat
        if np.all(mt.model == MODEL_J2):
            return j2_update(eps, self.eps_p, self.epbar, self.K, self.G, self.sy, self.H, self.n)
        sigma = np.zeros_like(eps)
        eps_p = self.eps_p.copy()
        epbar = self.epbar.copy()
        parts = []
        for model in (MODEL_J2, MODEL_NLELASTIC, MODEL_VISCO):
            m = mt.model == model
            if not np.any(m):
                continue
            e, ep, eb = eps[:, :, m], self.eps_p[:, :, m], self.epbar[m]
            if model == MODEL_J2:
                r = j2_update(e, ep, eb, mt.K[m], mt.G[m], mt.sy[m], mt.H[m], mt.n[m])
            elif model == MODEL_NLELASTIC:
                r = nonlinear_elastic_update(e, ep, eb, mt.K[m], mt.sy[m], mt.eps0[m], mt.n[m])
            else:
                r = visco_update(e, ep, eb, mt.K[m], mt.G[m], mt.sy[m], mt.eps0[m], mt.t0[m],
                                 mt.n[m], self.dt)
            sigma[:, :, m] = r.sigma
            eps_p[:, :, m] = r.eps_p
            epbar[m] = r.epbar
            parts.append((np.flatnonzero(m.reshape(-1)), r))
        return PointResult(sigma, eps_p, epbar, parts)


@dataclass
class StepResult:
    sigma: np.ndarray            # homogenised stress, 6 comps
    newton_iters: int
    cg_iters: int
    cg_per_newton: list
    residuals: list              # ||G sigma_i|| / ||sigma_i|| per Newton iteration
    newton_norms: list           # ||de_i|| / ||E||_field per Newton iteration
    converged: bool


def solve_increment(st: State, dE6, tol_newton, tol_cg, max_newton=50,
                    max_cg=2000, fixed_cg=None, fixed_newton=None, solver="cg"):
    """One increment of Algorithm 1 (increment loop body).

    E_t+dt = E_t + dE; Newton on G sigma(E + eps*) = 0 starting from the
    previous eps*; each Newton iteration solves G C de = -G sigma by CG;
    then one final constitutive call at the converged strain gives the
    homogenised stress (mean of the nodal stress, Eq. trapz) and the
    committed history. Updates `st` in place.
    """
    E = st.E + to_tensor(np.asarray(dE6, dtype=np.float64))
    eps_star = st.eps_star.copy()
    V = st.N ** 3
    normE = np.sqrt(V * np.sum(E * E))
    it = 0
    cg_total = 0
    cg_list, res_list, nn_list = [], [], []
    converged = False
    while True:
        res = st.constitutive(E, eps_star)
        Gs = project(res.sigma)
        nG = np.sqrt(inner(Gs, Gs))
        ns = np.sqrt(inner(res.sigma, res.sigma))
        res_list.append(nG / ns if ns > 0 else 0.0)
        tan = Tangent(res)
        if nG <= ROUNDOFF_RHS * ns:
            de, ncg = np.zeros_like(Gs), 0
        else:
            de, ncg, _ = linear_solve(solver, tan, res, -Gs, tol_cg, max_cg,
                                      ROUNDOFF_RHS * ns, fixed_iters=fixed_cg)
        eps_star += de
        it += 1
        cg_total += ncg
        cg_list.append(ncg)
        nde = np.sqrt(inner(de, de))
        rel = nde / normE if normE > 0 else (0.0 if nde == 0 else np.inf)
        nn_list.append(rel)
        if fixed_newton is not None:
            if it >= fixed_newton:
                converged = True
                break
            continue
        if rel <= tol_newton or nde == 0.0:
            converged = True
            break
        if it >= max_newton:
            break
    res = st.constitutive(E, eps_star)
    Sigma = to_comps(res.sigma.reshape(3, 3, -1).mean(axis=-1))
    if converged:
        st.E = E
        st.eps_star = eps_star
        st.eps_p = res.eps_p
        st.epbar = res.epbar
    return StepResult(Sigma, it, cg_total, cg_list, res_list, nn_list, converged)


def macro_tangent(st: State, tol_cg, max_cg=2000, solver="cg"):
    """6x6 algorithmic macroscopic tangent dSigma/dE at the committed state.

    Not in the paper. Column j perturbs tensor component j (a shear perturbs
    (i,j) and (j,i) together by 1): b_j = -G (C : E_j), solve G C de_j = b_j,
    C_hom[:, j] = mean(C : (E_j + de_j)). C is the tangent at the committed
    strain with the history of the previous increment (the trial state that
    produced the committed one), i.e. the last tangent of the increment.
    Requires `st.last_res`, which `solve_increment_keep` sets.
    """
    res = st.last_res
    tan = Tangent(res)
    N = st.N
    Ch = np.zeros((6, 6))
    for j, (a, b) in enumerate(PAIRS):
        Ej = np.zeros((3, 3))
        Ej[a, b] = 1.0
        Ej[b, a] = 1.0
        Ef = np.broadcast_to(Ej[:, :, None, None, None], (3, 3, N, N, N)).copy()
        CE = tan.apply(Ef)
        rhs = -project(CE)
        de, _, _ = linear_solve(solver, tan, res, rhs, tol_cg, max_cg,
                                ROUNDOFF_RHS * np.sqrt(inner(CE, CE)))
        s = tan.apply(Ef + de)
        Ch[:, j] = to_comps(s.reshape(3, 3, -1).mean(axis=-1))
    return Ch


def solve_increment_keep(st: State, dE6, tol_newton, tol_cg, **kw):
    """`solve_increment` that also keeps the final constitutive result.

    The last constitutive call is evaluated against the history of the
    previous increment, so it must be taken before the commit overwrites it.
    """
    eps_p_prev, epbar_prev = st.eps_p.copy(), st.epbar.copy()
    r = solve_increment(st, dE6, tol_newton, tol_cg, **kw)
    tmp = State(st.N, st.phase, st.mats, E=st.E, eps_star=st.eps_star,
                eps_p=eps_p_prev, epbar=epbar_prev, dt=st.dt)
    st.last_res = tmp.constitutive(st.E, st.eps_star)
    return r
