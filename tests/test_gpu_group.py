"""Increments of cells of several grid sizes as one CUDA graph launch
(fftg_group_*): the Newton loop of Algorithm 1 and each Newton iteration's
CG loop run on the device, the sizes' branches concurrently.

* The results equal, bit for bit, those of the host-driven batch step
  (fftg_batch_step) on identical handles: homogenised stress, Newton and
  CG counts, the committed strain field.
* A cell gives the same bits alone (a group of one one-cell handle) and in
  a group of cells of other grid sizes.
* FP64 group steps match the oracle (1e-10 in the homogenised stress,
  identical Newton and CG counts); cells left out by the run mask keep
  their state.
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


def _cells(spec, precision):
    """spec: [(N, [seeds])] -> phases, increments (a proportional path per cell)."""
    out = []
    for N, seeds in spec:
        ph = np.stack([I.random_spheres(N, 0.3, s, r_min=1.5, r_max=3.5)[0] for s in seeds])
        dE = np.stack([I.random_increment(100 + s, 1.5e-3) for s in seeds])
        out.append((N, ph, dE))
    return out


SPEC = [(9, [1, 2]), (15, [3, 4, 5]), (27, [6])]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_group_step_equals_batch_step_bit_for_bit(precision):
    cells = _cells(SPEC, precision)
    ga = [fftg.Cell(N, ph, I.TWO_PHASE, precision=precision, nrhs_tangent=0) for N, ph, _ in cells]
    gb = [fftg.Cell(N, ph, I.TWO_PHASE, precision=precision, nrhs_tangent=0) for N, ph, _ in cells]
    grp = fftg.Group(ga)
    for _ in range(3):
        res = grp.step([dE for _, _, dE in cells], 1e-5, 1e-8)
        for (N, ph, dE), cb, (sig, nn, nc, st) in zip(cells, gb, res):
            sb, nb, cgb, stb = cb.batch_step(dE, 1e-5, 1e-8)
            assert (st == 0).all() and (stb == 0).all()
            assert np.array_equal(sig, sb), (N, sig, sb)
            assert np.array_equal(nn, nb) and np.array_equal(nc, cgb)
    assert sum(int(c) for (_, nn, nc, _) in res for c in nc) > 0
    for ca, cb, (N, ph, _) in zip(ga, gb, cells):
        for k in range(ph.shape[0]):
            ca.select(k)
            cb.select(k)
            assert np.array_equal(ca.field(fftg.FFTG_FIELD_STRAIN), cb.field(fftg.FFTG_FIELD_STRAIN))
    assert grp.launch_count() > 0
    grp.close()
    for c in ga + gb:
        c.close()


def test_cell_alone_and_in_a_mixed_group_give_the_same_bits():
    cells = _cells(SPEC, "mixed")
    N, ph, dE = cells[2]
    alone = fftg.Cell(N, ph, I.TWO_PHASE, precision="mixed", nrhs_tangent=0)
    g1 = fftg.Group([alone])
    mixed = [fftg.Cell(n, p, I.TWO_PHASE, precision="mixed", nrhs_tangent=0) for n, p, _ in cells]
    g2 = fftg.Group(mixed)
    for _ in range(3):
        (s1, n1, c1, _), = g1.step([dE], 1e-5, 1e-8)
        r2 = g2.step([d for _, _, d in cells], 1e-5, 1e-8)
        s2, n2, c2, _ = r2[2]
        assert np.array_equal(s1, s2) and np.array_equal(n1, n2) and np.array_equal(c1, c2)
    g1.close()
    g2.close()
    for c in [alone] + mixed:
        c.close()


def test_fp64_group_matches_the_oracle_and_respects_the_run_mask():
    N = 15
    seeds = [11, 12]
    ph = np.stack([I.random_spheres(N, 0.3, s, r_min=2.0, r_max=4.0)[0] for s in seeds])
    path = I.shear_path(0.02, 20)
    cell = fftg.Cell(N, ph, I.TWO_PHASE, precision="fp64", nrhs_tangent=0)
    grp = fftg.Group([cell])
    sts = [O.State(N, ph[k], I.TWO_PHASE) for k in range(2)]
    for i in range(3):
        run = [np.array([1, 1 if i != 1 else 0])]       # the second cell skips increment 1
        (sig, nn, nc, st), = grp.step([np.stack([path[i], path[i]])], 1e-5, 1e-8, run=run)
        for k in range(2):
            if run[0][k] == 0:
                assert nn[k] == 0 and nc[k] == 0
                continue
            r = O.solve_increment(sts[k], path[i], 1e-5, 1e-8)
            assert np.abs(sig[k] - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()
            assert (nn[k], nc[k]) == (r.newton_iters, r.cg_iters)
    # the skipped cell is one increment behind: its committed E says so
    cell.select(1)
    eps = cell.field(fftg.FFTG_FIELD_STRAIN)
    assert abs(eps[5].mean() - 2 * path[0][5]) <= 1e-12
    grp.close()
    cell.close()
