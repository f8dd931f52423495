"""The basic scheme (Section 3.2, FFTG_SOLVER_RICHARDSON) on the GPU against
the oracle's Richardson iteration, and against the GPU's own CG.

Tolerances as in the other parity tests: FP64 solves 1e-10 in the
homogenised stress with identical Newton and iteration counts, mixed solves
1e-6; the reference-medium step comes from closed-form eigenvalues of the
compact tangent on the GPU and from a dense eigensolver in the oracle.
"""
import numpy as np
import pytest

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


def _cell9():
    N = 9
    ph, _, _ = I.random_spheres(N, 0.3, 5, r_min=1.5, r_max=3.0)
    return N, ph


def test_fp64_richardson_matches_oracle():
    N, ph = _cell9()
    st = O.State(N, ph, I.TWO_PHASE)
    cell = fftg.Cell(N, ph, I.TWO_PHASE, precision="fp64", solver="richardson", max_cg=20000)
    for dE in I.shear_path(0.0045, 3):
        r = O.solve_increment(st, dE, 1e-9, 1e-11, max_cg=20000, solver="richardson")
        sig, nn, nc = cell.step(dE, 1e-9, 1e-11)
        assert np.abs(sig - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()
        assert (nn, nc) == (r.newton_iters, r.cg_iters)
    assert nc > 0
    cell.close()


def test_mixed_richardson_reaches_the_fp64_result():
    N, ph = _cell9()
    st = O.State(N, ph, I.TWO_PHASE)
    cell = fftg.Cell(N, ph, I.TWO_PHASE, precision="mixed", solver="richardson", max_cg=20000)
    for dE in I.shear_path(0.0045, 3):
        r = O.solve_increment(st, dE, 1e-6, 1e-8)
        sig, nn, nc = cell.step(dE, 1e-6, 1e-8)
        assert cell.stats()["newton_norm"][-1] <= 1e-6
        assert np.abs(sig - r.sigma).max() <= 1e-6 * np.abs(r.sigma).max()
    cell.close()


def test_richardson_needs_more_iterations_than_cg_for_the_same_answer():
    N = 27
    ph, _, _ = I.random_spheres(N, 0.3, 8, r_min=2.0, r_max=4.0)
    out = {}
    for solver in ("cg", "richardson"):
        cell = fftg.Cell(N, ph, I.TWO_PHASE, precision="fp64", solver=solver, max_cg=20000)
        total = 0
        for dE in I.shear_path(0.0045, 3):
            sig, nn, nc = cell.step(dE, 1e-8, 1e-10)
            total += nc
        C, tc = cell.tangent(1e-10)
        out[solver] = (sig, total, C, tc)
        cell.close()
    assert np.abs(out["cg"][0] - out["richardson"][0]).max() <= 1e-8 * np.abs(out["cg"][0]).max()
    assert np.abs(out["cg"][2] - out["richardson"][2]).max() <= 1e-7 * np.abs(out["cg"][2]).max()
    assert out["richardson"][1] > 2 * out["cg"][1]
    assert out["richardson"][3] > 2 * out["cg"][3]
