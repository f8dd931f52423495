"""Pins of the oracle's DFT pair and projection against what the paper fixes.

Each test checks the oracle against something other than itself: a dense
DFT built from the definition, Parseval, a single Fourier mode, the
properties of Ghat stated in Section 2.2 and Appendix A, the independent
acoustic-tensor formula of Eq. (Gamma_explicit), and fields that are
compatible or equilibrated by construction (built with numpy's own
frequency table, not the oracle's).
"""
import numpy as np
import pytest

from oracle import fftg_oracle as O


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- DFT pair
@pytest.mark.parametrize("shape", [(5, 5, 5), (3, 5, 9), (1, 1, 1), (9, 3, 5), (15, 15, 15),
                                   (1, 1, 243), (1, 243, 1)])
@pytest.mark.parametrize("impl", ["library", "textbook"])
def test_dft_matches_dense_definition(shape, impl, monkeypatch):
    # both FFTs of the oracle against the dense DFT matrix, up to 15^3 and
    # along a 243-point axis (the benchmark's grid)
    monkeypatch.setattr(O, "FFT_IMPL", impl)
    t = _rng(1).standard_normal((2,) + shape)
    a = O.dft_forward(t)
    b = O.dft_forward_dense(t)
    assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())
    assert np.abs(O.dft_inverse(a).real - t).max() <= 1e-13 * np.abs(t).max()


@pytest.mark.parametrize("n", [2, 7, 11, 12, 49])
def test_textbook_fft_other_lengths(n):
    # the recursion is generic in the factors (prime lengths are summed
    # directly): compare with the DFT sum written out for a 1D signal
    x = _rng(n).standard_normal(n) + 1j * _rng(n + 1).standard_normal(n)
    m = np.arange(n)
    ref = np.exp(-2j * np.pi * np.outer(m, m) / n) @ x
    got = O.fft_textbook(x, axes=(-1,))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(45, 45, 45), (3, 5, 225), (1, 135, 81)])
def test_library_fft_matches_textbook_fft(shape):
    # past the sizes a dense matrix reaches, the library FFT the oracle uses
    # by default is pinned to the textbook mixed-radix recursion
    t = _rng(4).standard_normal(shape)
    a = np.fft.fftn(t, axes=(-3, -2, -1))
    b = O.fft_textbook(t)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_dft_roundtrip_parseval_and_single_mode():
    N = 15
    rng = _rng(2)
    t = rng.standard_normal((N, N, N))
    th = O.dft_forward(t)
    assert np.allclose(O.dft_inverse(th).real, t, atol=1e-13)
    # Parseval with the 1/|N| forward convention: sum |t|^2 = |N| sum |that|^2
    assert np.isclose((t * t).sum(), N ** 3 * (np.abs(th) ** 2).sum(), rtol=1e-12)
    # a single Fourier mode exp(2 pi i k.x/N) transforms to a unit delta at k
    k = (2, -3, 7)
    x = np.arange(N)
    ph = (k[0] * x[:, None, None] + k[1] * x[None, :, None] + k[2] * x[None, None, :]) / N
    mode = np.exp(2j * np.pi * ph)
    mh = O.dft_forward(mode)
    j = tuple(kk % N for kk in k)
    assert abs(mh[j] - 1.0) < 1e-12
    mh[j] = 0.0
    assert np.abs(mh).max() < 1e-12


def test_frequencies_reduced_index_set():
    for N in (1, 3, 5, 15, 27, 243):
        k = O.frequencies(N)
        assert np.array_equal(k, np.fft.fftfreq(N, d=1.0 / N).astype(int))
        assert k.max() == (N - 1) // 2 and k.min() == -((N - 1) // 2)


# ---------------------------------------------------------------- Ghat
def _random_xi(n=64, seed=3):
    xi = _rng(seed).standard_normal((n, 3))
    xi[0] = (1.0, 0.0, 0.0)
    xi[1] = (0.0, -2.0, 3.0)
    return xi


def test_ghat_idempotent_and_symmetric():
    g = O.ghat(_random_xi())
    gg = np.einsum("nijlm,nlmpq->nijpq", g, g)
    assert np.abs(gg - g).max() < 1e-14
    assert np.abs(g - g.transpose(0, 2, 1, 3, 4)).max() < 1e-15    # minor ij
    assert np.abs(g - g.transpose(0, 1, 2, 4, 3)).max() < 1e-15    # minor lm
    assert np.abs(g - g.transpose(0, 3, 4, 1, 2)).max() < 1e-15   # major


def test_ghat_zero_even_and_homogeneous():
    assert np.abs(O.ghat(np.zeros(3))).max() == 0.0
    xi = _random_xi()
    assert np.abs(O.ghat(-xi) - O.ghat(xi)).max() < 1e-15
    assert np.abs(O.ghat(2.5 * xi) - O.ghat(xi)).max() < 1e-14


def test_ghat_fixes_compatible_and_kills_equilibrated():
    rng = _rng(4)
    for xi in _random_xi(16):
        a = rng.standard_normal(3)
        comp = 0.5 * (np.outer(a, xi) + np.outer(xi, a))
        out = np.einsum("ijlm,lm->ij", O.ghat(xi), comp)
        assert np.abs(out - comp).max() < 1e-13 * np.abs(comp).max()
        n = xi / np.linalg.norm(xi)
        P = np.eye(3) - np.outer(n, n)
        A = rng.standard_normal((3, 3))
        eq = P @ (A + A.T) @ P            # tau n = 0
        out = np.einsum("ijlm,lm->ij", O.ghat(xi), eq)
        assert np.abs(out).max() < 1e-14 * np.abs(eq).max()


def test_ghat_equals_gamma_ref_with_symmetric_identity():
    # Appendix A: the two operators coincide for C_ref = I_s
    xi = _random_xi(128, seed=5)
    assert np.abs(O.ghat(xi) - O.gamma_ref(xi, O.I4s)).max() < 1e-14


def test_gamma_ref_differs_for_other_reference_media():
    # sanity of the pin itself: with a non-identity reference medium the
    # acoustic-tensor operator is not the projection
    Cref = 3.0 * O.II + 2.0 * O.I4s
    xi = _random_xi(8, seed=6)
    assert np.abs(O.ghat(xi) - O.gamma_ref(xi, Cref)).max() > 1e-2


# ---------------------------------------------------------------- G in real space
def _compatible_field(N, seed):
    """eps = sym grad u for a random periodic trig-polynomial displacement."""
    rng = _rng(seed)
    u = rng.standard_normal((3, N, N, N))
    uh = np.fft.fftn(u, axes=(1, 2, 3))
    k = np.fft.fftfreq(N, d=1.0 / N)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"))
    gh = 1j * np.einsum("ixyz,jxyz->ijxyz", K, uh)
    eh = 0.5 * (gh + gh.transpose(1, 0, 2, 3, 4))
    eps = np.fft.ifftn(eh, axes=(2, 3, 4))
    assert np.abs(eps.imag).max() < 1e-10
    return eps.real


def _equilibrated_field(N, seed):
    """tau with zero mean and tau(k) xi(k) = 0 at every frequency (div tau = 0)."""
    rng = _rng(seed)
    A = rng.standard_normal((3, 3, N, N, N))
    Ah = np.fft.fftn(A + A.transpose(1, 0, 2, 3, 4), axes=(2, 3, 4))
    k = np.fft.fftfreq(N, d=1.0 / N)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"))
    n2 = (K ** 2).sum(0)
    n2[0, 0, 0] = 1.0
    n = K / np.sqrt(n2)
    P = np.eye(3)[:, :, None, None, None] - np.einsum("ixyz,jxyz->ijxyz", n, n)
    th = np.einsum("ijxyz,jlxyz,lmxyz->imxyz", P, Ah, P)
    th[:, :, 0, 0, 0] = 0.0
    t = np.fft.ifftn(th, axes=(2, 3, 4))
    assert np.abs(t.imag).max() < 1e-10
    return t.real


@pytest.mark.parametrize("N", [5, 9, 15])
def test_projection_real_space_properties(N):
    eps = _compatible_field(N, 7)
    assert np.abs(O.project(eps) - eps).max() < 1e-12 * np.abs(eps).max()
    tau = _equilibrated_field(N, 8)
    assert np.abs(O.project(tau)).max() < 1e-12 * np.abs(tau).max()
    const = np.broadcast_to(np.arange(9.0).reshape(3, 3)[:, :, None, None, None] + 1,
                            (3, 3, N, N, N))
    const = 0.5 * (const + const.transpose(1, 0, 2, 3, 4))
    assert np.abs(O.project(const)).max() < 1e-13


def test_projection_self_adjoint_and_idempotent():
    N = 9
    rng = _rng(9)
    x = rng.standard_normal((3, 3, N, N, N)); x = x + x.transpose(1, 0, 2, 3, 4)
    y = rng.standard_normal((3, 3, N, N, N)); y = y + y.transpose(1, 0, 2, 3, 4)
    Gx, Gy = O.project(x), O.project(y)
    assert np.isclose(O.inner(Gx, y), O.inner(x, Gy), rtol=1e-12)
    assert np.abs(O.project(Gx) - Gx).max() < 1e-12 * np.abs(Gx).max()
    # G x + (I - G) x splits into compatible and equilibrated parts
    assert abs(O.inner(Gx, x - Gx)) < 1e-10 * O.inner(x, x)


def test_ghat_through_t_equals_appendix_a():
    # The fused P3 applies Ghat through t = tau n alone, as n(x)u + u(x)n
    # with u = t - (n.t / 2) n: the same operator as Appendix A's
    # Ghat_ijlm tau_lm (the oracle's explicit 3x3x3x3 array), for complex
    # symmetric tau and any xi != 0. Dropping the 1/2 breaks it.
    rng = _rng(21)
    for _ in range(50):
        xi = rng.integers(-121, 122, size=3).astype(np.float64)
        if not xi.any():
            continue
        a = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        tau = a + a.T
        ref = np.einsum("ijlm,lm->ij", O.ghat(xi), tau)
        n = xi / np.linalg.norm(xi)
        t = tau @ n
        u = t - 0.5 * (n @ t) * n
        got = np.outer(n, u) + np.outer(u, n)
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(tau).max()
        wrong = t - (n @ t) * n
        bad = np.outer(n, wrong) + np.outer(wrong, n)
        assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max() or np.abs(n @ t) < 1e-12
