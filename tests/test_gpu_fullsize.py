"""Parity at the benchmark's full size (243^3), in the launch configuration
the benchmark times.

The oracle cannot run a 243^3 solve, so these checks use what holds exactly
at any size:
* with a homogeneous elastic tangent C_e, a sum of Fourier modes maps to the
  sum of Ghat(k) : (C_e : A_k) on each mode (exact, evaluated with the
  oracle's Ghat per mode);
* with a heterogeneous plastic tangent, G C is symmetric on compatible
  fields and its output is compatible (G G C = G C); the FP32 result agrees
  with the FP64 one;
* a full load increment in mixed precision reaches the FP64 result.
"""
import numpy as np
import pytest

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 243


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_05970_gb300 import build
    build.build()
    fftg.load()


def _dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda").reshape(-1)


def _waves(nw, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(N, dtype=np.float64)
    modes = []
    for w in range(nw):
        k = rng.integers(-(N - 1) // 2, (N - 1) // 2 + 1, size=3)
        modes.append((k, rng.standard_normal(6), rng.uniform(0, 2 * np.pi)))
    def field(coef):
        out = np.zeros((6, N, N, N))
        for (k, A6, ph), c6 in zip(modes, coef):
            arg = (2 * np.pi / N) * (k[0] * x[:, None, None] + k[1] * x[None, :, None]
                                     + k[2] * x[None, None, :]) + ph
            cw = np.cos(arg)
            for c in range(6):
                out[c] += c6[c] * cw
        return out
    return modes, field


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_matvec_243_homogeneous_plane_waves_exact(prec):
    mat = I.Phase(0.833, 0.386, 1e9, 0.0)   # elastic everywhere: C = C_e
    cell = fftg.Cell(N, np.zeros((N, N, N), np.uint8), (mat,), precision=prec, nrhs_tangent=0)
    cell.constitutive()                       # tangent at zero strain: C_e
    modes, field = _waves(4, 3)
    Ce = mat.K * O.II + 2.0 * mat.G * O.I4d
    p = field([A6 for _, A6, _ in modes])
    ref = field([O.to_comps(np.einsum("ijlm,lm->ij", O.ghat(k.astype(float)),
                                      np.einsum("ijlm,lm->ij", Ce, O.to_tensor(A6))))
                 for k, A6, _ in modes])
    dt = torch.float64 if prec == "fp64" else torch.float32
    if prec == "mixed":
        p = p.astype(np.float32).astype(np.float64)
    q, _ = cell.matvec(_dev(p, dt))
    q = q.double().cpu().numpy().reshape(6, N, N, N)
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.linalg.norm(q - ref) <= tol * 3.0 * np.linalg.norm(p)
    cell.close()


def test_matvec_243_plastic_symmetric_compatible_and_fp32_matches_fp64():
    w = I.workload("spheres243")
    c64 = fftg.Cell(N, w["phase"], w["mats"], precision="fp64", nrhs_tangent=0)
    c32 = fftg.Cell(N, w["phase"], w["mats"], precision="mixed", nrhs_tangent=0)
    E = np.array([0.006, 0.0, 0.0, 0.0, 0.0, 0.002])   # most voxels plastic
    c64.constitutive(dE=E)
    c32.constitutive(dE=E)
    g = torch.Generator(device="cuda").manual_seed(7)
    xs = [c64.project(torch.randn(6 * N ** 3, dtype=torch.float64, device="cuda", generator=g))
          for _ in range(2)]
    x, y = xs
    Ax, _ = c64.matvec(x)
    Ay, _ = c64.matvec(y)
    # symmetry of G C on compatible fields (FP64), in the Frobenius product
    # (the shear components count twice)
    def frob(u, v):
        u6, v6 = u.view(6, -1), v.view(6, -1)
        return float((u6[:3] * v6[:3]).sum() + 2.0 * (u6[3:] * v6[3:]).sum())
    a, b = frob(y, Ax), frob(Ay, x)
    assert abs(a - b) <= 1e-11 * (abs(a) + abs(b))
    # the output is compatible: G (G C x) = G C x
    GAx = c64.project(Ax)
    assert float(torch.linalg.norm(GAx - Ax)) <= 1e-12 * float(torch.linalg.norm(Ax))
    # FP32 path against FP64
    Ax32, _ = c32.matvec(x.float())
    err = float(torch.linalg.norm(Ax32.double() - Ax)) / float(torch.linalg.norm(Ax))
    assert err <= 2e-5
    c64.close()
    c32.close()


def test_step_243_mixed_reaches_fp64_result():
    w = I.workload("spheres243")
    out = {}
    for prec in ("mixed", "fp64"):
        cell = fftg.Cell(N, w["phase"], w["mats"], precision=prec, nrhs_tangent=0)
        for dE in w["dE"][:4]:                 # two elastic, two plastic increments
            sig, nn, nc = cell.step(dE, w["tol_newton"], w["tol_cg"])
        out[prec] = sig
        st = cell.stats()
        assert st["newton_norm"][-1] <= w["tol_newton"]
        cell.close()
        torch.cuda.empty_cache()
    assert np.abs(out["mixed"] - out["fp64"]).max() <= 1e-6 * np.abs(out["fp64"]).max()
