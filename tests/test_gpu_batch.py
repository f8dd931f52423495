"""Batches of cells: one launch per pass for all cells, each cell with its own
Newton and CG iteration.

A cell's result must not depend on which other cells share its launches:
its reductions use per-cell partial sums in a fixed order, so the stress is
bit-identical alone and in a batch (the 'same alone and in the mix' check),
and it matches the FP64 oracle like any single cell.
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


def _phases(N, seeds, frac=0.3):
    return np.stack([I.random_spheres(N, frac, s, r_min=2.0, r_max=4.0)[0] for s in seeds])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_cells_alone_bitwise(prec):
    N = 15
    seeds = [11, 12, 13, 14]
    ph = _phases(N, seeds)
    dirs = np.stack([I.random_increment(100 + s, 1.0e-3) for s in seeds])
    batch = fftg.Cell(N, ph, I.TWO_PHASE, precision=prec, nrhs_tangent=0)
    alone = [fftg.Cell(N, ph[b], I.TWO_PHASE, precision=prec, nrhs_tangent=0) for b in range(4)]
    for inc in range(3):
        dE = dirs * (1.0 + 0.5 * inc)
        sig, nn, nc, st = batch.batch_step(dE, 1e-5, 1e-8)
        assert (st == 0).all()
        for b in range(4):
            s1, n1, c1 = alone[b].step(dE[b], 1e-5, 1e-8)
            assert np.array_equal(sig[b], s1), (prec, inc, b)
            assert (nn[b], nc[b]) == (n1, c1)
    batch.close()
    for c in alone:
        c.close()


def test_batch_fp64_matches_oracle_and_uneven_loading():
    N = 15
    seeds = [21, 22, 23]
    ph = _phases(N, seeds)
    batch = fftg.Cell(N, ph, I.TWO_PHASE, precision="fp64", nrhs_tangent=0)
    dE = np.zeros((3, 6))
    dE[0, 5] = 0.001         # shear
    dE[1, 0] = 0.0015        # uniaxial
    dE[2] = I.random_increment(7, 1e-3)
    sts = [O.State(N, ph[b], I.TWO_PHASE) for b in range(3)]
    for inc in range(3):
        sig, nn, nc, st = batch.batch_step(dE, 1e-5, 1e-8)
        assert (st == 0).all()
        for b in range(3):
            r = O.solve_increment(sts[b], dE[b], 1e-5, 1e-8)
            assert np.abs(sig[b] - r.sigma).max() <= 1e-10 * np.abs(r.sigma).max()
            assert (nn[b], nc[b]) == (r.newton_iters, r.cg_iters)
    # per-cell state access through select
    for b in range(3):
        batch.select(b)
        eps = batch.field(fftg.FFTG_FIELD_STRAIN)
        ref = O.to_comps(sts[b].eps_star) + O.to_comps(sts[b].E)[:, None, None, None]
        assert np.linalg.norm(eps - ref) <= 1e-9 * np.linalg.norm(ref)
    batch.close()


def test_batch_failed_cell_is_not_committed():
    N = 15
    ph = _phases(N, [31, 32])
    batch = fftg.Cell(N, ph, I.TWO_PHASE, precision="fp64", nrhs_tangent=0, max_newton=2)
    dE = np.zeros((2, 6))
    dE[:, 5] = 0.001
    batch.batch_step(dE, 1e-5, 1e-8)          # elastic: both converge at once
    batch.select(1)
    before = batch.get_state()
    dE2 = dE.copy()
    dE2[1, 5] = 0.01                          # a large plastic jump: Newton cap
    sig, nn, nc, st = batch.batch_step(dE2 * [[1], [1]], 1e-12, 1e-8)
    assert st[1] == fftg.FFTG_ENOCONV_NEWTON
    assert np.array_equal(batch.get_state(), before)
    batch.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_loop_equals_host_chunked_loop(prec):
    # the device-resident CG (graph with a conditional WHILE node) runs the
    # same kernels in the same order as the host-chunked loop: identical bits
    N = 27
    ph = _phases(N, [51, 52])
    a = fftg.Cell(N, ph, I.TWO_PHASE, precision=prec, nrhs_tangent=0, cg_graph=1)
    b = fftg.Cell(N, ph, I.TWO_PHASE, precision=prec, nrhs_tangent=0, cg_graph=0)
    dE = np.zeros((2, 6))
    dE[0, 5] = 0.0015
    dE[1, 0] = 0.0015
    for _ in range(3):
        ra = a.batch_step(dE, 1e-5, 1e-8)
        rb = b.batch_step(dE, 1e-5, 1e-8)
        assert np.array_equal(ra[0], rb[0])
        assert np.array_equal(ra[1], rb[1]) and np.array_equal(ra[2], rb[2])
    a.close()
    b.close()
