"""Continuous-batching server: results are the same alone and in the mix.

Several sessions share a server with fewer cells than sessions, so requests
join the running batch between Newton iterations and idle sessions are
evicted to host memory and restored. Every session's stress after every
increment must equal, bit for bit, the same sequence of increments run alone
on a single-cell handle: a cell's reductions never depend on what shares
its launches.
"""
import time

import numpy as np
import pytest

from paper_1601_05970_gb300 import fftg
from paper_1601_05970_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_05970_gb300 import build
    build.build()
    fftg.load()


def _collect(srv, n, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < n:
        for r in srv.poll(0.05):
            out[r["request_id"]] = r
        assert time.time() - t0 < timeout, "server did not finish"
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_server_same_alone_and_in_mix(prec):
    N = 15
    n_sess, n_inc = 4, 3
    phases = [I.random_spheres(N, 0.3, 40 + s, r_min=2.0, r_max=4.0)[0] for s in range(n_sess)]
    dE = [[I.random_increment(500 + 10 * s + k, 1.5e-3) for k in range(n_inc)] for s in range(n_sess)]
    # alone
    alone = {}
    for s in range(n_sess):
        cell = fftg.Cell(N, phases[s], I.TWO_PHASE, precision=prec, nrhs_tangent=0)
        for k in range(n_inc):
            alone[(s, k)] = cell.step(dE[s][k], 1e-5, 1e-8)[0]
        cell.close()
    # in the mix: 2 cells for 4 sessions, all requests submitted at once
    srv = fftg.Server(N, 2, I.TWO_PHASE, precision=prec, tol_newton=1e-5, tol_cg=1e-8)
    rid = 0
    ids = {}
    for k in range(n_inc):
        for s in range(n_sess):
            srv.submit(rid, s, dE[s][k], phases[s] if k == 0 else None)
            ids[rid] = (s, k)
            rid += 1
    res = _collect(srv, rid)
    info = srv.info()
    srv.stop()
    for r_id, r in res.items():
        assert r["status"] == 0
        assert np.array_equal(np.array(r["sigma"]), alone[ids[r_id]]), ids[r_id]
    # order within a session is submission order
    for s in range(n_sess):
        t = [res[i]["t_start"] for i in res if ids[i][0] == s]
        ks = [ids[i][1] for i in res if ids[i][0] == s]
        assert [k for _, k in sorted(zip(t, ks))] == list(range(n_inc))
    assert info["evictions"] > 0 and info["max_concurrent"] == 2


def test_server_admits_while_busy():
    # a request submitted while another is in flight joins the running batch
    N = 75
    ph = [I.random_spheres(N, 0.3, 60 + s)[0] for s in range(2)]
    srv = fftg.Server(N, 2, I.TWO_PHASE, precision="mixed")
    srv.submit(0, 0, [0, 0, 0, 0, 0, 0.004], ph[0])   # plastic: several Newton rounds
    time.sleep(0.002)
    srv.submit(1, 1, [0, 0, 0, 0, 0, 0.004], ph[1])
    res = _collect(srv, 2)
    info = srv.info()
    srv.stop()
    assert all(r["status"] == 0 for r in res.values())
    assert res[1]["t_start"] < res[0]["t_done"]       # started before the first finished
    assert info["max_concurrent"] == 2
