"""Seeded synthetic inputs: microstructures, material sets and load paths.

This module holds no arithmetic of the solver itself. It only produces the
inputs that both the CUDA path and the CPU oracle consume: phase maps (one
byte per voxel, x1 slowest, x3 fastest), per-phase J2 parameters and
macroscopic strain increments in the component order (11, 22, 33, 23, 13, 12)
of tensor (not engineering) strain components.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its
published definition so that the same seed gives the same microstructure on
any machine.

The periodic random-sphere generator stands in for the two-phase DP600
micrograph of the paper's Section 5.2, which is not available: it keeps the
paper's hard/soft two-phase structure and yield-stress ratio of 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1

# Component order of every 6-vector in this library: tensor components
# (11, 22, 33, 23, 13, 12); a shear entry is the tensor component, not the
# engineering strain.
COMPONENTS = ("11", "22", "33", "23", "13", "12")


class SplitMix64:
    """SplitMix64 counter-based generator (Steele et al. 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def gaussian(self) -> float:
        """Standard normal by the Box-Muller transform."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


# Constitutive models of Section 4 (the `model` entry of a material tuple)
MODEL_J2, MODEL_NLELASTIC, MODEL_VISCO = 0, 1, 2


@dataclass(frozen=True)
class Phase:
    """J2 material with isotropic hardening sigma_0 + H epbar^n (Section 4.2;
    n = 1 is linear hardening)."""

    K: float        # bulk modulus
    G: float        # shear modulus
    sigma_y: float  # initial yield stress sigma_0
    H: float        # hardening modulus
    n: float = 1.0  # hardening exponent (> 0)

    def as_tuple(self):
        """(K, G, sigma_0, H, n, eps_0, t_0, model), the field order of the
        library's phase record."""
        return (self.K, self.G, self.sigma_y, self.H, self.n, 0.0, 0.0, MODEL_J2)


@dataclass(frozen=True)
class NonlinearElastic:
    """Non-linear elastic material of Section 4.1:
    sigma = K tr(eps) I + sigma_0 (eps_eq / eps_0)^n N."""

    K: float        # bulk modulus
    sigma0: float   # reference stress sigma_0
    eps0: float     # reference strain eps_0
    n: float        # exponent

    def as_tuple(self):
        return (self.K, 0.0, self.sigma0, 0.0, self.n, self.eps0, 0.0, MODEL_NLELASTIC)


@dataclass(frozen=True)
class ViscoPlastic:
    """Visco-plastic material of Section 4.3 (Norton's rule
    gamma_dot = (eps_0 / t_0) (sigma_eq / sigma_0)^(1/n)) with the elasticity
    of Section 4.2."""

    K: float        # bulk modulus
    G: float        # shear modulus
    sigma0: float   # reference stress sigma_0
    eps0: float     # reference strain eps_0
    t0: float       # reference time t_0
    n: float        # strain-rate sensitivity exponent

    def as_tuple(self):
        return (self.K, self.G, self.sigma0, 0.0, self.n, self.eps0, self.t0, MODEL_VISCO)


def material_tuple(m):
    """The 8-entry tuple (K, G, sigma_0, H, n, eps_0, t_0, model) of a material
    given as an object with as_tuple() or as (K, G, sigma_y, H[, n]) (J2)."""
    t = tuple(float(v) for v in (m.as_tuple() if hasattr(m, "as_tuple") else m))
    if len(t) == 4:
        t = t + (1.0,)
    if len(t) == 5:
        t = t + (0.0, 0.0, float(MODEL_J2))
    if len(t) != 8:
        raise ValueError(f"material {m!r}: expected 4, 5 or 8 entries")
    return t


# The two-phase material set used by every workload: bulk 0.833, shear 0.386,
# soft matrix (phase 0) yield 0.003 / hardening 0.01, hard phase (phase 1)
# yield 0.006 / hardening 0.02 (yield and hardening ratio 2 as in Section 5.2).
@dataclass(frozen=True)
class SaintVenantKirchhoff:
    """Hyperelastic phase of the finite-strain path: W = lambda/2 (tr E)^2
    + mu E : E with the Green-Lagrange strain E = (F^T F - I)/2. Its
    small-strain limit is isotropic elasticity with K = lambda + 2 mu/3,
    G = mu."""

    lam: float
    mu: float

    def as_tuple(self):
        return (self.lam, self.mu)


SOFT = Phase(K=0.833, G=0.386, sigma_y=0.003, H=0.01)
HARD = Phase(K=0.833, G=0.386, sigma_y=0.006, H=0.02)
TWO_PHASE = (SOFT, HARD)
# Finite strain: the elastic constants of SOFT and a phase five times stiffer
SVK_SOFT = SaintVenantKirchhoff(lam=0.833 - 2.0 * 0.386 / 3.0, mu=0.386)
SVK_HARD = SaintVenantKirchhoff(lam=5.0 * (0.833 - 2.0 * 0.386 / 3.0), mu=5.0 * 0.386)
SVK_TWO_PHASE = (SVK_SOFT, SVK_HARD)


def check_grid(N: int) -> None:
    """Odd N of the form 3^a 5^b (Section 2.3: odd grids only)."""
    if N < 1 or N % 2 == 0:
        raise ValueError(f"N={N}: the grid must have an odd number of nodes")
    m = N
    for p in (3, 5):
        while m % p == 0:
            m //= p
    if m != 1:
        raise ValueError(f"N={N}: only products of 3 and 5 are supported")


def laminate(N: int, n_hard: int, axis: int = 0) -> np.ndarray:
    """Two-phase laminate: phase 1 where the index along `axis` is < n_hard."""
    ph = np.zeros((N, N, N), dtype=np.uint8)
    sl = [slice(None)] * 3
    sl[axis] = slice(0, n_hard)
    ph[tuple(sl)] = 1
    return ph


def random_spheres(N: int, fraction: float, seed: int,
                   r_min: float = 3.0, r_max: float = 8.0):
    """Periodic random hard spheres in a soft matrix.

    Centres are uniform in [0, N)^3 (continuous), radii uniform in
    [r_min, r_max]; voxel (i, j, l), located at integer coordinates, is hard
    when its minimum-image distance to a centre is at most the radius.
    Spheres are added until the hard fraction reaches `fraction`.
    Returns (phase map uint8 [N,N,N], achieved fraction, number of spheres).
    """
    rng = SplitMix64(seed)
    ph = np.zeros(N ** 3, dtype=np.uint8)
    target = int(math.ceil(fraction * N ** 3))
    count = 0
    nsph = 0
    if fraction <= 0.0:
        return ph.reshape(N, N, N), 0.0, 0
    while count < target:
        c = [rng.uniform() * N for _ in range(3)]
        r = r_min + (r_max - r_min) * rng.uniform()
        nsph += 1
        axes = []
        idx = []
        for d in range(3):
            g = np.arange(int(math.floor(c[d] - r)), int(math.ceil(c[d] + r)) + 1)
            delta = g - c[d]
            delta = delta - N * np.round(delta / N)
            axes.append(delta)
            idx.append(np.mod(g, N))
        d2 = (axes[0][:, None, None] ** 2 + axes[1][None, :, None] ** 2
              + axes[2][None, None, :] ** 2)
        inside = d2 <= r * r
        lin = (idx[0][:, None, None] * N + idx[1][None, :, None]) * N + idx[2][None, None, :]
        flat = np.unique(lin[inside])
        new = int(np.count_nonzero(ph[flat] == 0))
        ph[flat] = 1
        count += new
    return ph.reshape(N, N, N), count / N ** 3, nsph


def shear_path(gamma_max: float, n_inc: int) -> np.ndarray:
    """Pure shear E = gamma (e1 x e2 + e2 x e1), ramped linearly (Eq. shear_strain).

    Returns the per-increment macroscopic strain increments [n_inc, 6].
    """
    dE = np.zeros((n_inc, 6))
    dE[:, 5] = gamma_max / n_inc
    return dE


def uniaxial_path(e11_max: float, n_inc: int) -> np.ndarray:
    """Uniaxial strain: only E11 is non-zero, ramped linearly."""
    dE = np.zeros((n_inc, 6))
    dE[:, 0] = e11_max / n_inc
    return dE


def stretch_shear_path(n_inc: int) -> np.ndarray:
    """Finite-strain load path: n_inc equal increments dF of the macroscopic
    deformation gradient, [n_inc, 3, 3]; each stretches x1 by 1 %, shears
    (F12) by 0.5 % and contracts x2 and x3 by 0.4 %."""
    dF = np.array([[0.01, 0.005, 0.0], [0.0, -0.004, 0.0], [0.0, 0.0, -0.004]])
    return np.repeat(dF[None], n_inc, axis=0)


def frobenius6(v) -> float:
    """Frobenius norm of a symmetric tensor given as 6 components."""
    v = np.asarray(v, dtype=np.float64)
    return float(math.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2
                           + 2.0 * (v[3] ** 2 + v[4] ** 2 + v[5] ** 2)))


def random_increment(seed: int, norm: float = 1e-3) -> np.ndarray:
    """Random symmetric strain increment with Frobenius norm `norm`.

    The direction is a seeded Gaussian on the 6 components; each shear entry
    stands for both (i, j) and (j, i), so it enters the norm twice.
    """
    rng = SplitMix64(seed)
    v = np.array([rng.gaussian() for _ in range(6)])
    return v * (norm / frobenius6(v))


def workload(name: str, seed: int | None = None):
    """Named workloads with their sizes (see the docstrings of the generators).

    Returns a dict with keys N, phase (uint8 [N,N,N]), mats (tuple of Phase),
    dE (increments [n, 6]), tol_newton, tol_cg and a description. `seed`
    replaces the microstructure seed of the random-sphere workloads.
    """
    if name == "laminate15":
        N = 15
        return dict(N=N, phase=laminate(N, 5, axis=0), mats=TWO_PHASE,
                    dE=shear_path(0.02, 10), tol_newton=1e-5, tol_cg=1e-8,
                    desc="15^3 two-phase laminate (hard where x1-index < 5), "
                         "pure shear to 0.02 in 10 increments")
    if name == "spheres135":
        N = 135
        seed = 1 if seed is None else seed
        ph, frac, _ = random_spheres(N, 0.3, seed=seed)
        return dict(N=N, phase=ph, mats=TWO_PHASE, dE=shear_path(0.02, 20),
                    tol_newton=1e-5, tol_cg=1e-8, fraction=frac, seed=seed,
                    desc=f"135^3 random spheres r in [3,8], hard fraction 0.3, "
                         f"seed {seed}, pure shear to 0.02 in 20 increments")
    if name == "spheres243":
        N = 243
        seed = 2 if seed is None else seed
        ph, frac, _ = random_spheres(N, 0.2, seed=seed)
        return dict(N=N, phase=ph, mats=TWO_PHASE, dE=uniaxial_path(0.03, 20),
                    tol_newton=1e-5, tol_cg=1e-8, fraction=frac, seed=seed,
                    desc=f"243^3 random spheres r in [3,8], hard fraction 0.2, "
                         f"seed {seed}, uniaxial strain E11 to 0.03 in 20 increments")
    if name in ("fs_spheres135", "fs_spheres243"):
        N = int(name[len("fs_spheres"):])
        seed = 2 if seed is None else seed
        ph, frac, _ = random_spheres(N, 0.2, seed=seed)
        return dict(N=N, phase=ph, mats=SVK_TWO_PHASE, dF=stretch_shear_path(20),
                    tol_newton=1e-6, tol_cg=1e-8, fraction=frac, seed=seed,
                    desc=f"{N}^3 random spheres r in [3,8], hard fraction 0.2, seed {seed}, "
                         f"St. Venant-Kirchhoff phases (hard 5x soft), F11 to 1.2 with "
                         f"F12 to 0.1 and lateral contraction in 20 increments")
    raise KeyError(name)
