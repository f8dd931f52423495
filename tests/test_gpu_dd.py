"""The double-float FFTs of the mixed path's residual (FFTG_DD) against the
oracles' projections.

Double-float numbers carry about 48 significant bits (rounding near 2^-47,
7e-15), and a 3D FFT pair adds some tens of such roundings, each relative
to the norm of its operands: the bound used is 1e-12 of the largest entry,
about a hundred times the expected error and ten times below the CG roundoff
floor (1e-13 of the norm, summed over the grid). FP32 FFTs miss it by five
orders of magnitude (checked below, so the test would see a fall-back).
"""
import numpy as np
import pytest

from oracle import fftg_finite_strain as FS
from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_05970_gb300 import build
    build.build()
    fftg.load()


@pytest.mark.parametrize("N", [5, 15, 45, 81])
def test_small_strain_projection_in_double_float(N):
    rng = np.random.default_rng(100 + N)
    tau = rng.standard_normal((6, N, N, N))
    ref = O.to_comps(O.project(O.to_tensor(tau)))
    cell = fftg.Cell(N, np.zeros((N, N, N), np.uint8), (I.SOFT,), precision="mixed", nrhs_tangent=0)
    t = torch.tensor(tau.reshape(-1), device="cuda")
    out = cell.project(t, dd=True).cpu().numpy().reshape(tau.shape)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err <= 1e-12, err
    out32 = cell.project(t.float()).cpu().double().numpy().reshape(tau.shape)
    assert np.abs(out32 - ref).max() / np.abs(ref).max() > 1e-9
    cell.close()


@pytest.mark.parametrize("N", [15, 45, 75])
def test_finite_strain_projection_in_double_float(N):
    rng = np.random.default_rng(200 + N)
    A = rng.standard_normal((3, 3, N, N, N))
    ref = FS.project_fs(A)
    cell = fftg.FsCell(N, np.zeros((N, N, N), np.uint8), (I.SVK_SOFT,), precision="mixed")
    out = cell.project(torch.tensor(A.reshape(-1), device="cuda"), dd=True).cpu().numpy().reshape(A.shape)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err <= 1e-12, err
    cell.close()


def test_double_float_projection_at_243_is_idempotent_and_keeps_the_mean_out():
    # the grid of the bench's residual passes: properties that hold at any size
    N = 243
    rng = np.random.default_rng(7)
    tau = torch.tensor(rng.standard_normal(6 * N ** 3) + 3.0, device="cuda")   # with a mean
    cell = fftg.Cell(N, np.zeros((N, N, N), np.uint8), (I.SOFT,), precision="mixed", nrhs_tangent=0)
    g = cell.project(tau, dd=True)
    gg = cell.project(g, dd=True)
    scale = g.abs().max().item()
    assert (gg - g).abs().max().item() <= 1e-12 * scale
    assert g.view(6, -1).mean(dim=1).abs().max().item() <= 1e-13 * scale
    cell.close()
