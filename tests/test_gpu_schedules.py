"""Every schedule the autotuner can choose (radix split and tile of the FP32
passes of the mixed CG iteration) against the FP64 oracle, and the tuner
itself.

For each grid size, pass kind and schedule variant (the others at their
defaults, every handle created after the schedule is set):
* the FP32 projection G tau against the oracle's, to 2e-5 of |tau| (the
  FP32 operator tolerance of the other parity tests);
* one plastic increment of the mixed solver against the oracle's
  homogenised stress, to 1e-6 relative (the mixed-precision tolerance).
Then the tuner: it times every variant, keeps a valid choice per pass, and
a second call with the cache file reads the choice back without timing.
"""
import numpy as np
import pytest

from oracle import fftg_oracle as O
from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E0 = np.array([0, 0, 0, 0, 0, 0.002])
DE = np.array([0, 0, 0, 0, 0, 0.001])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_05970_gb300 import build
    build.build()
    fftg.load()
    yield
    for N in (27, 45):
        for k in fftg.SCHED_KINDS:
            fftg.schedule_set(N, k, 0)


_REF = {}


def _reference(N):
    if N not in _REF:
        ph, _, _ = I.random_spheres(N, 0.3, 5, r_min=2.0, r_max=4.0)
        tau = np.random.default_rng(N).standard_normal((6, N, N, N)).astype(np.float32).astype(np.float64)
        g = O.to_comps(O.project(O.to_tensor(tau)))
        st = O.State(N, ph, I.TWO_PHASE, E=O.to_tensor(E0))
        r = O.solve_increment(st, DE, 1e-5, 1e-8)
        assert (st.epbar > 0).mean() > 0.05
        _REF[N] = (ph, tau, g, r.sigma)
    return _REF[N]


@pytest.mark.parametrize("N", [27, 45])
@pytest.mark.parametrize("kind", list(fftg.SCHED_KINDS))
def test_every_schedule_matches_the_oracle(N, kind):
    ph, tau, gref, sref = _reference(N)
    for v in range(fftg.SCHED_VARIANTS):
        for k in fftg.SCHED_KINDS:
            fftg.schedule_set(N, k, 0)
        fftg.schedule_set(N, kind, v)
        assert fftg.schedule_get(N)[kind] == v
        cell = fftg.Cell(N, ph, I.TWO_PHASE, precision="mixed", nrhs_tangent=0)
        out = cell.project(torch.tensor(tau.reshape(-1), dtype=torch.float32, device="cuda"))
        out = out.double().cpu().numpy().reshape(6, N, N, N)
        assert np.linalg.norm(out - gref) <= 2e-5 * np.linalg.norm(tau), (kind, v)
        cell.set_state(np.concatenate([E0, np.zeros(13 * N ** 3)]))
        sig, nn, nc = cell.step(DE, 1e-5, 1e-8)
        assert nc > 0
        assert np.abs(sig - sref).max() <= 1e-6 * np.abs(sref).max(), (kind, v)
        cell.close()
    fftg.schedule_set(N, kind, 0)


def test_schedule_shapes_are_distinct_where_the_grid_allows():
    # 243 = 27 x 9: the other split is 9 x 27; P3's tile halves (variant 2)
    # or stays the default one with stage B, Ghat and the inverse stage B in
    # one phase (variant 3)
    d0 = fftg.schedule_describe(243, "p3", 0)
    d1 = fftg.schedule_describe(243, "p3", 1)
    assert d0["split"] == (27, 9) and d1["split"] == (9, 27)
    assert fftg.schedule_describe(243, "p3", 2)["cols"] * 2 == d0["cols"]
    assert fftg.schedule_describe(243, "p3", 3) == d0
    r0 = fftg.schedule_describe(243, "p1", 0)["rows"]
    assert fftg.schedule_describe(243, "p1", 2)["rows"] * 2 == r0
    assert fftg.schedule_describe(27, "p2", 1)["split"] == (9, 3)


def test_autotune_picks_a_schedule_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setenv("FFTG_SCHEDULE_CACHE", str(tmp_path / "sched.txt"))
    chosen, ms = fftg.autotune(27, cache=True)
    assert set(chosen) == set(fftg.SCHED_KINDS)
    for k, v in chosen.items():
        assert 0 <= v < fftg.SCHED_VARIANTS
        assert all(t > 0 for t in ms[k])
        # a variant replaces the default only when 2 % faster
        assert 0.98 * ms[k][v] <= min(ms[k]) * (1 + 1e-9)
        assert fftg.schedule_get(27)[k] == v
    for k in fftg.SCHED_KINDS:
        fftg.schedule_set(27, k, 0)
    again, ms2 = fftg.autotune(27, cache=True)
    assert again == chosen and all(t == -1.0 for k in ms2 for t in ms2[k])
    assert fftg.schedule_get(27) == chosen
    # the tuned schedules still solve to the oracle's stress
    ph, tau, gref, sref = _reference(27)
    cell = fftg.Cell(27, ph, I.TWO_PHASE, precision="mixed", nrhs_tangent=0)
    cell.set_state(np.concatenate([E0, np.zeros(13 * 27 ** 3)]))
    sig, nn, nc = cell.step(DE, 1e-5, 1e-8)
    assert np.abs(sig - sref).max() <= 1e-6 * np.abs(sref).max()
    cell.close()
    for k in fftg.SCHED_KINDS:
        fftg.schedule_set(27, k, 0)


@pytest.mark.parametrize("N", [135, 243])
def test_fused_p3_matches_the_default_at_full_size(N):
    """P3 variant 3 (stage B, Ghat and the inverse stage B in one phase, t =
    tau n accumulated over the components) sums in another order than the
    default tile, so G tau agrees with it to FP32 rounding at the full grid
    sizes (the default's G tau is checked against the oracle at these sizes
    in the full-size tests)."""
    rng = np.random.default_rng(7 + N)
    ph = np.zeros((N, N, N), dtype=np.int8)
    tau = rng.standard_normal(6 * N ** 3).astype(np.float32)
    out = {}
    for v in (0, 3):
        fftg.schedule_set(N, "p3", v)
        cell = fftg.Cell(N, ph, I.TWO_PHASE, precision="mixed", nrhs_tangent=0)
        out[v] = cell.project(torch.tensor(tau, device="cuda")).cpu().numpy().astype(np.float64)
        cell.close()
    fftg.schedule_set(N, "p3", 0)
    assert np.isfinite(out[3]).all()
    assert np.linalg.norm(out[3] - out[0]) <= 1e-6 * np.linalg.norm(out[0])
    assert np.abs(out[3] - out[0]).max() <= 1e-5 * np.abs(out[0]).max()
