"""The seeded input generators (paper_1601_05970_gb300/inputs.py): the
counter-based generator against published values, and the structure of the
synthetic microstructures and load paths the tests and the benchmark use."""
import numpy as np

from paper_1601_05970_gb300 import inputs as I


def test_splitmix64_published_sequence():
    # SplitMix64 (Steele, Lea and Flood 2014) from state 0: the first
    # outputs as published with the reference implementation
    g = I.SplitMix64(0)
    assert g.next_u64() == 0xE220A8397B1DCDAF
    assert g.next_u64() == 0x6E789E6AA1B965F4
    assert g.next_u64() == 0x06C45D188009454F


def test_uniform_is_in_unit_interval_and_roughly_flat():
    g = I.SplitMix64(7)
    u = np.array([g.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=10, range=(0.0, 1.0))
    assert np.abs(hist / len(u) - 0.1).max() < 0.01


def test_random_spheres_reach_the_fraction_and_are_periodic_and_seeded():
    N = 45
    ph, frac, nsph = I.random_spheres(N, 0.3, seed=3)
    assert ph.shape == (N, N, N) and ph.dtype == np.uint8
    assert set(np.unique(ph)) <= {0, 1}
    assert 0.3 <= frac < 0.3 + 0.05 and abs(ph.mean() - frac) < 1e-12
    assert nsph > 1
    ph2, frac2, _ = I.random_spheres(N, 0.3, seed=3)
    assert np.array_equal(ph, ph2) and frac == frac2          # same seed, same map
    ph3, _, _ = I.random_spheres(N, 0.3, seed=4)
    assert not np.array_equal(ph, ph3)
    # minimum-image distances: a sphere near the boundary wraps around
    ph_b, _, _ = I.random_spheres(9, 0.5, seed=1, r_min=2.0, r_max=3.0)
    assert ph_b[0].any() and ph_b[-1].any()


def test_laminate_and_load_paths():
    ph = I.laminate(15, 5, axis=0)
    assert ph[:5].all() and not ph[5:].any()
    sp = I.shear_path(0.02, 10)
    assert sp.shape == (10, 6) and np.allclose(sp.sum(axis=0)[:5], 0.0)
    fs = I.stretch_shear_path(20)
    assert fs.shape == (20, 3, 3)
    Fbar = np.eye(3) + fs.sum(axis=0)
    assert np.allclose(Fbar, [[1.2, 0.1, 0.0], [0.0, 0.92, 0.0], [0.0, 0.0, 0.92]])


def test_finite_strain_phases_have_the_small_strain_elastic_constants():
    # the soft St. Venant-Kirchhoff phase linearises to the J2 phases'
    # elasticity: K = lambda + 2 mu / 3, G = mu
    m = I.SVK_SOFT
    assert abs(m.lam + 2.0 * m.mu / 3.0 - I.SOFT.K) < 1e-15 and m.mu == I.SOFT.G
    assert I.SVK_HARD.lam == 5.0 * m.lam and I.SVK_HARD.mu == 5.0 * m.mu
