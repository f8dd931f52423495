"""Request driver for the continuous-batching servers (fftg_server_*).

An FE^2 macro solver issues RVE increments as its Gauss points need them.
This driver stands in for it: Poisson arrivals at a given rate, each request
one increment of Frobenius norm 1e-3 for one session (an RVE with its own
microstructure and history), the grid size of the session drawn with given
weights. Each session follows its own proportional strain path (a seeded
random direction), as a Gauss point under monotone macroscopic loading
does, so its history accumulates plastic strain from request to request. One server per grid size runs its own
worker thread and stream, so the sizes overlap on the GPU; each server's
cell count comes from its share of the HBM budget. `run` reports solves
per second and latency percentiles (submit to result, on the servers'
clock).
"""
from __future__ import annotations

import math
import threading
import time

import numpy as np

from . import fftg
from . import inputs as I


def slots_for_budget(N, budget_bytes, precision="mixed", max_slots=32):
    """Cells of grid N that fit in `budget_bytes` of device memory (at least
    one, at most max_slots), and the bytes of one more cell."""
    opt = fftg.default_options()
    opt.precision = fftg.FFTG_MIXED if precision == "mixed" else fftg.FFTG_FP64
    opt.nrhs_tangent = 0
    lib = fftg.load()
    import ctypes as C
    one = C.c_size_t(0)
    fftg.check(lib.fftg_workspace_size_batch(N, 1, C.byref(opt), C.byref(one)), "size")
    two = C.c_size_t(0)
    fftg.check(lib.fftg_workspace_size_batch(N, 2, C.byref(opt), C.byref(two)), "size")
    per = max(1, two.value - one.value)
    base = one.value - per
    n = int((budget_bytes - base) // per)
    return max(1, min(max_slots, n)), per


def session_microstructure(N, session_id):
    """Random hard spheres (radii 3-8, periodic) with a hard fraction drawn in
    [0.1, 0.4], both seeded by the session id."""
    rng = I.SplitMix64(10_000 + session_id)
    frac = 0.1 + 0.3 * rng.uniform()
    ph, got, _ = I.random_spheres(N, frac, seed=20_000 + session_id)
    return ph


def run(rate, duration, Ns=(27, 45, 75, 135), weights=(0.4, 0.3, 0.2, 0.1),
        sessions_per_N=None, budget_gb=None, precision="mixed", seed=5,
        tol_newton=1e-5, tol_cg=1e-8, max_requests=None, drain_s=None, max_slots=64,
        mem_fraction=0.5):
    """Poisson arrivals for `duration` seconds at `rate` requests/s.

    Device memory: `budget_gb`, or by default `mem_fraction` of the device
    memory free at the start, split between the grid sizes in proportion to
    their request weights times their footprint per cell, so that each size
    gets cells in proportion to its share of the requests (at most
    `max_slots` per size). A request is admitted when a cell of its size is
    free; a resident idle session is evicted to host memory only when every
    cell of the size is taken.

    After the arrivals stop, requests still queued get `drain_s` seconds
    (default: `duration`) to be admitted; then the queues are cancelled and
    the requests in flight finish. Above the servers' capacity that backlog
    is reported (`backlog`, `saturated`), and a latency percentile that the
    cancelled requests would decide is reported as None.

    Returns a dict with solves/s, p50/p95/p99 latency (ms), per-size counts
    and server statistics.
    """
    import torch
    weights = np.asarray(weights, dtype=float) / np.sum(weights)
    if budget_gb is None:
        free, _ = torch.cuda.mem_get_info()
        budget = mem_fraction * free
    else:
        budget = budget_gb * 1e9
    per_cell = {N: slots_for_budget(N, 0, precision)[1] for N in Ns}
    wb = sum(w * per_cell[N] for N, w in zip(Ns, weights))
    servers, slot_info = {}, {}
    for N, w in zip(Ns, weights):
        slots, per = slots_for_budget(N, budget * w * per_cell[N] / wb, precision, max_slots)
        servers[N] = fftg.Server(N, slots, I.TWO_PHASE, precision=precision,
                                 tol_newton=tol_newton, tol_cg=tol_cg)
        slot_info[N] = dict(slots=slots, bytes_per_slot=per)
    if sessions_per_N is None:
        # the workload's session pool: 64 RVEs (Gauss points) per grid size,
        # each following its own strain path, so the work per request
        # (elastic at first, plastic after a few increments) does not depend
        # on the memory. A session's increments run one after another, so
        # the pool also bounds the requests of a size in flight at once.
        sessions_per_N = {N: 64 for N in Ns}
    # sessions and microstructures are made before the clock starts
    sess = {}
    sid = 0
    for N in Ns:
        for _ in range(sessions_per_N[N]):
            sess[sid] = (N, session_microstructure(N, sid))
            sid += 1
    by_N = {N: [k for k, v in sess.items() if v[0] == N] for N in Ns}
    created = set()

    rng = np.random.default_rng(seed)
    n_req = int(rate * duration * 1.2) + 16
    gaps = rng.exponential(1.0 / rate, size=n_req)
    sizes = rng.choice(len(Ns), size=n_req, p=weights)
    picks = rng.random(n_req)

    results = []
    lock = threading.Lock()
    stop = threading.Event()

    def collector():
        while not stop.is_set() or any(len(pending[N]) for N in Ns):
            got_any = False
            for N, srv in servers.items():
                for r in srv.poll(0.0):
                    with lock:
                        results.append(r)
                        pending[N].discard(r["request_id"])
                    got_any = True
            if not got_any:
                time.sleep(0.0005)

    pending = {N: set() for N in Ns}
    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = fftg.Server.clock()
    t_next = t0
    submitted = 0
    for i in range(n_req):
        t_next += gaps[i]
        if t_next - t0 > duration or (max_requests and submitted >= max_requests):
            break
        while True:
            now = fftg.Server.clock()
            if now >= t_next:
                break
            time.sleep(min(0.002, t_next - now))
        N = Ns[sizes[i]]
        pool = by_N[N]
        s_id = pool[int(picks[i] * len(pool))]
        dE = I.random_increment(1_000_000 + s_id, 1e-3)
        phase = None
        if s_id not in created:
            phase = sess[s_id][1]
            created.add(s_id)
        with lock:
            pending[N].add(i)
        servers[N].submit(i, s_id, dE, phase)
        submitted += 1
    t_sub_end = fftg.Server.clock()
    drain = duration if drain_s is None else drain_s
    while fftg.Server.clock() - t_sub_end < drain:
        with lock:
            if not any(len(pending[N]) for N in Ns):
                break
        time.sleep(0.01)
    cancelled = 0
    for N, srv in servers.items():
        c = srv.cancel_pending()
        cancelled += c
    # the cancelled requests give no result: the collector stops waiting
    # for them once only they are left
    t_cancel = fftg.Server.clock()
    while True:
        with lock:
            n_left = sum(len(pending[N]) for N in Ns)
        if n_left <= cancelled or fftg.Server.clock() - t_cancel > 120.0:
            break
        time.sleep(0.01)
    with lock:
        for N in Ns:
            pending[N].clear()
    stop.set()
    th.join()
    t_end = fftg.Server.clock()
    infos = {N: srv.info() for N, srv in servers.items()}
    for srv in servers.values():
        srv.stop()
    lat = np.array([r["t_done"] - r["t_submit"] for r in results]) * 1e3
    ok = sum(1 for r in results if r["status"] == 0)
    # a percentile is known when the cancelled requests (latency above any
    # completed one) cannot reach it
    total = len(results) + cancelled

    def pct(q):
        if not lat.size:
            return None
        if cancelled == 0:
            return float(np.percentile(lat, q))
        rank = int(math.ceil(q / 100.0 * total))   # nearest rank among all requests
        return float(np.sort(lat)[rank - 1]) if rank <= lat.size else None
    per_N = {}
    for N in Ns:
        l = np.array([r["t_done"] - r["t_submit"] for r in results if sess[r["session_id"]][0] == N]) * 1e3
        cgs = [r["cg_iters"] for r in results if sess[r["session_id"]][0] == N]
        per_N[N] = dict(count=int(l.size), p50_ms=float(np.percentile(l, 50)) if l.size else None,
                        p99_ms=float(np.percentile(l, 99)) if l.size else None,
                        mean_cg_iters=float(np.mean(cgs)) if cgs else None,
                        slots=slot_info[N]["slots"], sessions=sessions_per_N[N],
                        evictions=infos[N]["evictions"], max_concurrent=infos[N]["max_concurrent"],
                        mean_batch=round(infos[N]["mean_batch"], 2))
    return dict(rate=rate, duration_s=round(t_sub_end - t0, 3), requests=submitted,
                completed=len(results), ok=ok, backlog=cancelled, saturated=cancelled > 0,
                solves_per_s=len(results) / max(t_end - t0, 1e-9),
                p50_ms=pct(50), p95_ms=pct(95), p99_ms=pct(99),
                per_N=per_N, precision=precision, budget_gb=round(budget / 1e9, 1))


def batched_workload(n_rve=256, Ns=(15, 27, 45, 75), seed=1000):
    """Seeded RVE set: N uniform over Ns, hard fraction uniform in [0.1, 0.4],
    each RVE with its own microstructure seed (seed + i) and its own
    proportional strain path (one random direction of norm 1e-3 per
    increment)."""
    rng = I.SplitMix64(seed)
    rves = []
    for i in range(n_rve):
        N = Ns[min(len(Ns) - 1, int(rng.uniform() * len(Ns)))]
        frac = 0.1 + 0.3 * rng.uniform()
        ph, _, _ = I.random_spheres(N, frac, seed=seed + i)
        rves.append(dict(N=N, phase=ph, dE=I.random_increment(seed + i, 1e-3), frac=frac))
    return rves


def run_batched(rves, n_inc=5, precision="mixed", tol_newton=1e-5, tol_cg=1e-8, graph=True):
    """All RVEs of one grid size form one batch handle (one launch per pass
    for the whole group of that size).

    graph=True: the handles of all sizes form one fftg_group, and each
    increment of every RVE is ONE CUDA graph launch (Newton and CG loops on
    the device, the sizes' branches concurrent). graph=False: each size is
    driven from its own host thread and stream (a host round trip per Newton
    iteration). Returns RVE solves/s and per-size counts."""
    import torch
    groups = {}
    for i, r in enumerate(rves):
        groups.setdefault(r["N"], []).append(i)
    cells, streams = {}, {}
    for N, idx in groups.items():
        streams[N] = torch.cuda.Stream()
        ph = np.stack([rves[i]["phase"] for i in idx])
        cells[N] = fftg.Cell(N, ph, I.TWO_PHASE, precision=precision, nrhs_tangent=0,
                             stream=streams[N])
    out = {N: dict(cells=len(idx), newton=0, cg=0, failed=0, seconds=0.0) for N, idx in groups.items()}
    if graph:
        Ns = sorted(groups)
        grp = fftg.Group([cells[N] for N in Ns])
        dEs = [np.stack([rves[i]["dE"] for i in groups[N]]) for N in Ns]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_inc):
            res = grp.step(dEs, tol_newton, tol_cg)
            for N, (sig, nn, nc, st) in zip(Ns, res):
                out[N]["newton"] += int(nn.sum())
                out[N]["cg"] += int(nc.sum())
                out[N]["failed"] += int((st != 0).sum())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        launches = grp.launch_count()
        grp.close()
        for c in cells.values():
            c.close()
        n = len(rves) * n_inc
        return dict(rves=len(rves), increments=n_inc, solves=n, seconds=wall, solves_per_s=n / wall,
                    groups={str(N): v for N, v in sorted(out.items())}, precision=precision,
                    mode="one graph launch per increment for all sizes", graph_launches=n_inc,
                    kernel_launches=launches)

    def work(N):
        idx = groups[N]
        dE = np.stack([rves[i]["dE"] for i in idx])
        t0 = time.perf_counter()
        for _ in range(n_inc):
            sig, nn, nc, st = cells[N].batch_step(dE, tol_newton, tol_cg)
            out[N]["newton"] += int(nn.sum())
            out[N]["cg"] += int(nc.sum())
            out[N]["failed"] += int((st != 0).sum())
        torch.cuda.synchronize()
        out[N]["seconds"] = time.perf_counter() - t0

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ths = [threading.Thread(target=work, args=(N,)) for N in groups]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    for c in cells.values():
        c.close()
    n = len(rves) * n_inc
    return dict(rves=len(rves), increments=n_inc, solves=n, seconds=wall,
                solves_per_s=n / wall, groups={str(N): v for N, v in sorted(out.items())},
                precision=precision, mode="one host thread and stream per size")


def main(argv=None):
    """Rate sweep: one JSON line per Poisson rate (requests/s)."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description="continuous-batching RVE serving sweep")
    ap.add_argument("--rates", default="50,100,200,500")
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--budget-gb", type=float, default=None,
                    help="device memory for the cells (default: half of the free memory)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args(argv)
    fftg.load()
    for rate in [float(r) for r in args.rates.split(",")]:
        res = run(rate, args.seconds, budget_gb=args.budget_gb, precision=args.precision)
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
