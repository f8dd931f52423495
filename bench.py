#!/usr/bin/env python
"""Benchmark of the FFT-Galerkin Newton-CG solver on one or more GB300s.

Workload: the 243^3 periodic cell with random hard spheres (radii 3-8,
hard fraction 0.2, seed 2), J2 with linear hardening, mixed precision (FP32
inner CG, FP64 return mapping, residual and homogenisation), on the load
path of that workload: uniaxial strain E11 to 0.03 in 20 increments of
0.0015 (Newton-CG to 1e-5 / CG 1e-8, FP32 inner floor 1e-5), then the 6x6
macroscopic tangent (six right-hand sides in one batched CG).

A timed step is one increment of that path, from E11 = 0; the 6x6 tangent
at the end of the K timed increments is timed too, so that --steps 20 times
the whole path with its tangent (K <= 20). The warm-up increments run on the
same cell, which is then reset to the undeformed state.

Metric: CG-iteration voxels/s = N^3 x (CG iterations of the Newton solves +
CG iterations of the six tangent solves) / device time of the timed region.
The line also carries the FE^2 pair (one increment + the 6x6 tangent) at the
end of the path, the plain FP64 path at 243^3 with its FP64 arithmetic
roofline, the roofline of the dominant kernel, of the matvec and of the
whole CG iteration, and the oracle timed on the host cores.

With --gpus N under torchrun each rank solves its own cell (own seed): the
path shards by cell with no data exchange (replicas; weak scaling).
`--impl reference` times the FP64 numpy oracle on the host cores instead.
"""
import os

# the oracle legs run one numpy thread per process (each process is counted
# as one of `cores`)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import concurrent.futures as cf
import json
import multiprocessing as mp
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG-iter voxels/s at 243^3 (FP32-inner vs plain FP64)"
UNIT = "voxel-iterations/s"
PATH_INCREMENTS = 20          # the workload's load path: E11 to 0.03 in 20 increments


# Algorithmic bytes per voxel and per field of each kernel kind (what the
# kernel must read and write given its interface; FP32 fields are 24 B per
# voxel, the half spectrum 6 x (H/N) x 8 B, the compact tangent 28 B; FP64
# twice that).
def bytes_per_voxel(N):
    H = (N + 1) // 2
    s32 = 6 * 8 * H / N
    s64 = 2 * s32
    return {
        # r, p, x in; p, x out; tangent; spectrum out (steady state: the
        # first iteration of a solve reads no p or x)
        "p1_cg_f32": 5 * 24 + 28 + s32,
        "p2_f32": 2 * s32, "p3_f32": 2 * s32, "p4_f32": 2 * s32,
        "p5_dot_f32": s32 + 24 + 24,               # spectrum in; q out; p in
        "cg_update_f32": 3 * 24,                   # r, q in; r out
        # the mixed path's CG without the update pass: P1 as p1_cg (and the
        # dot <p, C:p>), P5 reads the spectrum and r and writes r
        "p1_cgf_f32": 5 * 24 + 28 + s32,
        "p5_cgf_f32": s32 + 24 + 24,
        "cg_rr_f32": 0.0,                          # block partials only
        "p1_tanrhs_f32": 28 + s32,
        "p5_rhs_f32_to_f32": s32 + 24,
        "p1_cg_f64": 5 * 48 + 56 + s64,
        "p2_f64": 2 * s64, "p3_f64": 2 * s64, "p4_f64": 2 * s64,
        "p5_dot_f64": s64 + 48 + 48, "cg_update_f64": 3 * 48,
        "p1_plain_f64": 48 + s64,
        "p5_rhs_f64_to_f32": s64 + 24,
    }


# The CG kernels of one iteration, in launch order: with the update pass
# (FP64 path, basic scheme) and without it (mixed path).
CG_KINDS = ("p1_cg", "p2", "p3", "p4", "p5_dot", "cg_update")
MATVEC_KINDS = ("p1_cg", "p2", "p3", "p4", "p5_dot")
CGF_KINDS = ("p1_cgf", "p2", "p3", "p4", "p5_cgf", "cg_rr")

# Pencil plans N = N1 x N2 of the FFT passes (the register DFT of N1 points,
# then of N2 points).
PLANS = {3: (3, 1), 5: (5, 1), 9: (9, 1), 15: (15, 1), 25: (25, 1), 27: (27, 1), 45: (9, 5),
         75: (15, 5), 81: (9, 9), 125: (25, 5), 135: (15, 9), 225: (15, 15), 243: (27, 9)}
# real flops of a radix-3 and a radix-5 butterfly and of a complex product
_BF = {3: 16, 5: 48}
_CMUL = 6


def _regdft_flops(R):
    """Flops of the R-point register DFT: split R = P Q (P the smallest of 3
    and 5 dividing R), Q butterflies of P points, (P-1)(Q-1) non-trivial
    twiddles, P DFTs of Q points."""
    if R == 1:
        return 0
    P = 3 if R % 3 == 0 else 5
    Q = R // P
    return Q * _BF[P] + (P - 1) * (Q - 1) * _CMUL + P * _regdft_flops(Q)


def fft_flops(N):
    """Flops of one complex N-point pencil transform of the passes: stage A
    (N2 DFTs of N1 points, then the (N1-1)(N2-1) non-trivial twiddles),
    stage B (N1 DFTs of N2 points)."""
    N1, N2 = PLANS[N]
    return N2 * _regdft_flops(N1) + (N1 - 1) * (N2 - 1) * _CMUL + N1 * _regdft_flops(N2)


def flops_per_voxel(N):
    """Algorithmic flops per voxel and per field of the CG kernels, counted
    on the algorithm the kernels implement (any precision): the pencil FFTs
    (three complex transforms per row of six real components in P1/P5, six
    per column in P2-P4, two directions in P3), the real-to-complex split
    and merge (8 and 4 flops per pair and frequency), C : p with the compact
    tangent (41), Ghat in closed form (93 per frequency, six components), the
    CG vector updates (12 per update of six components) and dots (12)."""
    H = (N + 1) // 2
    F = fft_flops(N)
    row = 3 * F / N                       # three complex pencils per row of N voxels
    col = 6 * H * F / N ** 2              # six components x H x N pencils per N^3 voxels
    return {
        "p1_cg": 24 + 41 + row + 24 * H / N,
        "p2": col, "p4": col,
        "p3": 2 * col + 93 * H / N,
        "p5_dot": 12 * H / N + row + 12,
        "cg_update": 12 + 12,
    }



# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the dominant kernels from one ncu capture each (the ncu summaries kept
# with the repository give the command), valid while the kernel sources
# have the digest they had then (SHA-256 prefix of the files listed).
KERNEL_FILES = ("common.cuh", "fft_core.cuh", "passes.cuh")
FS_KERNEL_FILES = KERNEL_FILES + ("fs_passes.cuh",)
TRAFFIC = {"p1_cgf_f32": {"N": 243, "bytes": 2413.6e6, "digest": "82255a5e31b86c10", "files": KERNEL_FILES},
           "fs_p1_cgf_f32": {"N": 243, "bytes": 3587.1e6, "digest": "43f6874074ac81bb", "files": FS_KERNEL_FILES}}


def _strip_comments(src: bytes) -> bytes:
    """C++ source without // and /* */ comments and blank lines (string
    literals in these kernel headers hold no comment markers)."""
    import re
    text = src.decode()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(l.rstrip() for l in text.splitlines() if l.strip()).encode()


def kernel_digest(files=KERNEL_FILES):
    """SHA-256 prefix of the kernel sources with their comments removed:
    any change of code invalidates a traffic capture, a comment edit does
    not."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1601_05970_gb300", "csrc", f), "rb") as fh:
            h.update(_strip_comments(fh.read()))
    return h.hexdigest()[:16]


def measured_traffic(kind, N):
    """The captured DRAM bytes per launch of `kind` at N^3, or None when the
    kernel sources have changed since the capture."""
    tr = TRAFFIC.get(kind)
    if tr and tr["N"] == N and tr["digest"] == kernel_digest(tr["files"]):
        return tr["bytes"]
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--N", type=int, default=243)
    ap.add_argument("--no-tangent", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 comparison, the batched and the serving runs")
    ap.add_argument("--no-graph", action="store_true",
                    help="enqueue CG iterations from the host instead of the graph loop")
    ap.add_argument("--no-tune", action="store_true",
                    help="run the default schedules of the FP32 passes (no autotuning)")
    ap.add_argument("--projection-only", action="store_true",
                    help="time the FP32 projection G tau of a random field on a bare cell of "
                         "grid --N (the five passes alone, default schedules) and print it")
    ap.add_argument("--finite-strain-only", action="store_true",
                    help="run only the finite-strain line (mixed, --N 243 or 135) and print it")
    ap.add_argument("--serve-rates", default="50,100,200,500",
                    help="Poisson request rates (requests/s) of the serving runs")
    ap.add_argument("--serve-seconds", type=float, default=6.0)
    return ap.parse_args()


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------- oracle legs
# The oracle as it stands (FP64 numpy, one thread per process), timed on the
# host cores: each job times a fixed number of CG iterations (G C p on full
# 3x3 tensors and the vector updates) on a cell whose tangent comes from one
# stress update at the macroscopic strain the timed GPU increments pass
# through (E11 = 0.0045, no history). Jobs run in spawned processes, started
# before the first CUDA call.
_ORACLE_CELL = {}


def _oracle_cell(N_full, seed, sub, corner):
    """Tangent and right-hand side of the sub^3 block at `corner` of the
    N_full^3 workload (periodic closure), kept per process across calls."""
    key = (N_full, seed, sub, corner)
    if key not in _ORACLE_CELL:
        from oracle import fftg_oracle as O
        from paper_1601_05970_gb300 import inputs as I
        _ORACLE_CELL.clear()
        if N_full in (243, 135):
            w = I.workload(f"spheres{N_full}", seed=seed)
            ph, mats = w["phase"], w["mats"]
        else:
            ph, _, _ = I.random_spheres(N_full, 0.3, seed=seed)
            mats = I.TWO_PHASE
        c = corner
        ph = np.ascontiguousarray(np.roll(ph, (-c, -c, -c), axis=(0, 1, 2))[:sub, :sub, :sub])
        st = O.State(sub, ph, mats)
        res = st.constitutive(O.to_tensor(np.array([0.0045, 0, 0, 0, 0, 0])),
                              np.zeros((3, 3, sub, sub, sub)))
        rng = np.random.default_rng(seed + corner)
        b = O.to_tensor(rng.standard_normal((6, sub, sub, sub)))
        _ORACLE_CELL[key] = (O.Tangent(res), b)
    return _ORACLE_CELL[key]


def oracle_job(N_full, seed, n_iters, sub, corner=0):
    """One timed oracle run: n_iters CG iterations (fixed count) on the
    sub^3 block. Returns (voxel-iterations, t_start, t_end) on the host's
    wall clock (time.time, comparable across processes)."""
    from oracle import fftg_oracle as O
    tan, b = _oracle_cell(N_full, seed, sub, corner)
    t0 = time.time()
    O.cg(lambda p: O.matvec(tan, p), b, 1e-30, fixed_iters=n_iters)
    t1 = time.time()
    return sub ** 3 * n_iters, t0, t1


def oracle_pool(workers):
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def oracle_all_cores(pool, cores, N_full, seed, n_iters=2, sub=63):
    """`cores` single-threaded oracle runs at once, each on its own block of
    the workload: the aggregate is the work of all runs over the span from
    the first start to the last end."""
    futs = [pool.submit(oracle_job, N_full, seed, n_iters, sub, 27 * k) for k in range(cores)]
    res = [f.result() for f in futs]
    units = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return units / span


def oracle_per_n(pool, Ns=(15, 27, 45, 75, 135), seed=7):
    """Single-threaded oracle CG-iteration voxels/s on full N^3 cells of
    random spheres (the sizes of the batched and serving workloads and of
    the 135^3 shear workload), one job per N, run one after another."""
    out = {}
    for N in Ns:
        n_it = int(min(20, max(1, 2e6 // N ** 3)))
        units, t0, t1 = pool.submit(oracle_job, N, seed if N != 135 else 1, n_it, N, 0).result()
        out[str(N)] = units / (t1 - t0)
    return out


def run_reference(args):
    """The oracle as the reference arm: each step is one oracle CG iteration
    on every host core at once (one single-threaded process per core, each
    on its own 63^3 block of the 243^3 workload); the value is the aggregate
    CG-iteration voxels/s."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    sub = 63
    pool = oracle_pool(cores)
    # set-up of every process's block (stress update, tangent), untimed
    list(pool.map(oracle_job, *zip(*[(args.N, 2, 1, sub, 27 * k) for k in range(cores)])))
    vals, spans = [], []
    for k in range(args.warmup + args.steps):
        v = oracle_all_cores(pool, cores, args.N, 2, n_iters=1, sub=sub)
        if k >= args.warmup:
            vals.append(v)
    pool.shutdown()
    value = float(np.mean(vals))
    ms = 1e3 * cores * sub ** 3 / value
    desc = (f"FP64 numpy oracle, one CG iteration per step (G C p on full 3x3 tensors and the "
            f"vector updates) on each of {cores} {sub}^3 blocks of the {args.N}^3 workload "
            f"(seed 2, tangent at E11 = 0.0045), one single-threaded process per host core")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"spheres{args.N}-uniaxial (oracle blocks of {sub}^3)", "N": args.N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- ranks
def rank_seed(rank, base=2):
    """Each rank solves its own cell: the microstructure seed of rank r
    (base: the workload's own seed, 2 at 243^3 and 1 at 135^3)."""
    return base + 1000 * rank


def reduce_over_ranks(dist, dev_ms, wall_ms, units, launches, device):
    """Job time = the slowest rank (max); work = the sum over ranks. Only the
    timing is exchanged: the ranks' cells share no data."""
    import torch
    t = torch.tensor([dev_ms, wall_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units, float(launches)], device=device, dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(u[0]), int(u[1])


# --------------------------------------------------------------- extras
def precision_lines(N, fma64=None, precisions=("mixed", "fp64"), n_inc=4, timed_from=2):
    """The two precisions on the same plastic increments: fresh cells (no
    tangent) of the N^3 workload run increments 0..n_inc-1 of its load path;
    increments timed_from.. (plastic) are timed with CUDA events and on the
    host clock, with the library's per-kernel events on. Returns per
    precision the time to converged stress, the CG-iteration voxels/s of
    those increments and the per-kernel table, the speedup of mixed over
    FP64 and their difference in the homogenised stress. The FP64 entry
    carries the FP64 arithmetic roofline of its CG iteration against the
    measured FP64 FMA rate `fma64` (TFLOP/s)."""
    import torch
    from paper_1601_05970_gb300 import fftg
    from paper_1601_05970_gb300 import inputs as I
    w = I.workload("spheres243" if N == 243 else "spheres135")
    V = N ** 3
    out = {}
    sig_ref = None
    for prec in precisions:
        cell = fftg.Cell(N, w["phase"], w["mats"], precision=prec, nrhs_tangent=0)
        stream = cell.stream
        iters, wall, dev = [], 0.0, 0.0
        for k in range(n_inc):
            if k == timed_from:
                cell.profile(True)
                cell.profile_reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            t0 = time.perf_counter()
            sig, nn, nc = cell.step(w["dE"][k], w["tol_newton"], w["tol_cg"])
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= timed_from:
                wall += time.perf_counter() - t0
                dev += e0.elapsed_time(e1) * 1e-3
                iters.append((nn, nc))
        prof = cell.profile_read()
        cg = sum(c for _, c in iters)
        newton = sum(n for n, _ in iters)
        o = dict(seconds=wall, device_s=dev, increments=n_inc - timed_from, newton_cg=iters,
                 cg_iter_voxels_per_s=V * cg / dev, sigma=[float(v) for v in sig])
        sfx = "_f32" if prec == "mixed" else "_f64"
        # P2-P4 also run once per Newton iteration: the projection of the
        # FP32 inner solution (mixed) or the FP64 residual (FP64)
        rf = cg_roofline(prof, N, cg, newton, 0, sfx)
        o["kernels"] = rf["kernels"]
        o["iteration_ms"] = rf["iteration"]["ms_per_field_iter"]
        if prec == "fp64" and fma64:
            fl = sum(flops_per_voxel(N).values())
            tf = fl * V / (rf["iteration"]["ms_per_field_iter"] * 1e-3) / 1e12
            o["roofline"] = {"bound": "alu", "what": "FP64 CG iteration (P1-P5 + update)",
                             "achieved": tf, "peak": fma64, "unit": "TFLOP/s", "frac": tf / fma64,
                             "flops_per_voxel": fl, "peak_source": "measured FP64 FMA rate "
                             "(fftg_probe_fma_rate) in this run",
                             "hbm_frac": rf["iteration"]["frac"]}
        out[prec] = o
        if sig_ref is None:
            sig_ref = sig
        else:
            o["max_rel_diff_sigma_vs_" + precisions[0]] = float(
                np.abs(sig - sig_ref).max() / np.abs(sig_ref).max())
        cell.close()
        del cell
        torch.cuda.empty_cache()
    if "mixed" in out and "fp64" in out:
        out["speedup_mixed_over_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


def cg_roofline(prof, N, field_iters, projections, tangent_calls, sfx="_f32", hbm=None):
    """HBM roofline of the CG kernels from the library's per-kernel event
    times `prof` ({kind: (ms, launches)}): per kernel, the device time per
    field launch (a launch covers every field of a batch; launches of a
    finished solve return at entry and are not counted), the algorithmic
    bytes per voxel and the achieved fraction of the copy bandwidth; the
    same for the matvec (P1-P5) and the whole iteration (+ update).

    Field launches: the CG kernels run once per CG field-iteration; P2-P4
    of the inner precision also run `projections` more times (once per
    Newton iteration: the projection of an FP32 inner solution in the mixed
    path, the FP64 residual in the FP64 path) and, per tangent, once per
    right-hand side (six) and, in FP32, once per projection of its six
    solutions."""
    if hbm is None:
        hbm, _ = measured_hbm()
    bpv = bytes_per_voxel(N)
    V = N ** 3
    fused = ("p1_cgf" + sfx) in prof
    kinds, mv_kinds = (CGF_KINDS, CGF_KINDS[:5]) if fused else (CG_KINDS, MATVEC_KINDS)
    eff = {k: field_iters for k in ("p1_cg", "p5_dot", "cg_update", "p1_cgf", "p5_cgf", "cg_rr")}
    for k in ("p2", "p3", "p4"):
        eff[k] = field_iters + projections + (12 if sfx == "_f32" else 6) * tangent_calls
    kern = {}
    for base in kinds:
        name = base + sfx
        if name not in prof or not eff[base]:
            continue
        ms = prof[name][0] / eff[base]
        b = bpv[name]
        gbs = b * V / (ms * 1e-3) / 1e9
        kern[base] = {"ms": round(ms, 4), "bytes_per_voxel": round(b, 1), "GB/s": round(gbs, 1),
                      "frac": round(gbs / hbm, 3)}
    if fused and "cg_rr" not in kern:          # older builds: the reduction ran in P5
        kinds = kinds[:5]

    def agg(kinds, what):
        if not all(k in kern for k in kinds):
            return None
        ms = sum(kern[k]["ms"] for k in kinds)
        b = sum(kern[k]["bytes_per_voxel"] for k in kinds)
        gbs = b * V / (ms * 1e-3) / 1e9
        return {"what": what, "ms_per_field_iter": round(ms, 4), "bytes_per_voxel": round(b, 1),
                "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 3)}

    return {"kernels": kern,
            "matvec": agg(mv_kinds, "P1-P5: q = G(C:p) with the fused CG steps, per field"),
            "iteration": agg(kinds, "one CG iteration, per field: P1-P5" +
                             (" (update fused into P1/P5)" if fused else " + update pass"))}


def basic_scheme_line(N=135, n_inc=4, timed_from=2):
    """The basic scheme of Section 3.2 (Richardson's iteration with the
    reference medium (lambda_min + lambda_max)/2 I_s) against CG on the
    same cell and load path: linear-solver iterations and wall time of the
    plastic increments, mixed precision, fresh cells (no tangent)."""
    import torch
    from paper_1601_05970_gb300 import fftg
    from paper_1601_05970_gb300 import inputs as I
    w = I.workload("spheres135")
    out = {"N": N, "workload": "spheres135-uniaxial", "precision": "mixed"}
    for solver in ("cg", "richardson"):
        cell = fftg.Cell(N, w["phase"], w["mats"], precision="mixed", nrhs_tangent=0,
                         solver=solver, max_cg=20000)
        t_tot, iters = 0.0, []
        for k in range(n_inc):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sig, nn, nc = cell.step(w["dE"][k], w["tol_newton"], w["tol_cg"])
            torch.cuda.synchronize()
            if k >= timed_from:
                t_tot += time.perf_counter() - t0
                iters.append((nn, nc))
        out[solver] = dict(seconds=t_tot, newton_iters=[a for a, _ in iters],
                           solver_iters=[b for _, b in iters], sigma=[float(v) for v in sig])
        cell.close()
        del cell
        torch.cuda.empty_cache()
    out["iteration_ratio"] = sum(out["richardson"]["solver_iters"]) / max(1, sum(out["cg"]["solver_iters"]))
    out["time_ratio"] = out["richardson"]["seconds"] / out["cg"]["seconds"]
    return out


def fs_bytes_per_voxel(N):
    """Algorithmic bytes per voxel of the finite-strain CG kernels (FP32
    fields of nine components, 36 B per voxel; half spectrum 9 x (H/N) x 8 B;
    the tangent data is H = F - I, 36 B, and the phase byte)."""
    H = (N + 1) // 2
    s32 = 9 * 8 * H / N
    return {"fs_p1_cg_f32": 5 * 36 + 36 + 1 + s32,
            "fs_p2_f32": 2 * s32, "fs_p3_f32": 2 * s32, "fs_p4_f32": 2 * s32,
            "fs_p5_dot_f32": s32 + 36 + 36, "fs_cg_update_f32": 3 * 36,
            # without the update pass: P1 as above (and <p, K:p>); P5 reads
            # the spectrum and r and writes r
            "fs_p1_cgf_f32": 5 * 36 + 36 + 1 + s32, "fs_p5_cgf_f32": s32 + 36 + 36,
            "fs_cg_rr_f32": 0.0}


def projection_line(N, steps, warmup):
    """G tau of a random FP32 field on a bare mixed cell of grid N (one
    phase, no tangent RHS: a small device footprint), the five passes with
    their default schedules: ms per projection between CUDA events on the
    cell's stream, and the library's per-kernel times."""
    import torch
    from paper_1601_05970_gb300 import fftg
    from paper_1601_05970_gb300 import inputs as I
    cell = fftg.Cell(N, np.zeros((N, N, N), dtype=np.int8), I.TWO_PHASE, precision="mixed", nrhs_tangent=0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(N)
    tau = torch.randn(6 * N ** 3, device="cuda", generator=gen)
    out = torch.empty_like(tau)
    with torch.cuda.stream(cell.stream):
        for _ in range(max(1, warmup)):
            cell.project(tau, out)
        cell.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cell.stream)
        for _ in range(steps):
            cell.project(tau, out)
        e1.record(cell.stream)
        e1.synchronize()
    prof = cell.profile_read()
    cell.profile(False)
    cell.close()
    return {"what": "FP32 projection G tau, five passes (P1 plain, P2, P3, P4, P5 plain), default schedules",
            "N": N, "projections": steps, "ms_per_projection": e0.elapsed_time(e1) / max(1, steps),
            "kernels": {k: {"ms_per_launch": ms / max(1, n), "launches": n} for k, (ms, n) in prof.items()}}


def finite_strain_line(N=243, warm=1, timed=2):
    """The finite-strain extension (St. Venant-Kirchhoff, first
    Piola-Kirchhoff stress, gradient projection) on the N^3 spheres cell
    (243 or 135), mixed precision. One step is an increment of the
    stretch-shear path plus the 9x9 macroscopic tangent (the FE^2 call
    pair); steps warm.. are timed with CUDA events and per-kernel events,
    and the roofline is that of the dominant kernel."""
    import torch
    from paper_1601_05970_gb300 import fftg
    from paper_1601_05970_gb300 import inputs as I
    w = I.workload(f"fs_spheres{N}")
    N = w["N"]
    V = N ** 3
    cell = fftg.FsCell(N, w["phase"], w["mats"], precision="mixed")
    for k in range(warm):
        cell.step(w["dF"][k], w["tol_newton"], w["tol_cg"])
        cell.tangent(w["tol_cg"])
    cell.profile(True)
    stream = cell.stream
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = cell.launches()
    ev0.record(stream)
    t0 = time.perf_counter()
    nn_tot = nc_tot = nt_tot = 0
    for k in range(warm, warm + timed):
        P, nn, nc = cell.step(w["dF"][k], w["tol_newton"], w["tol_cg"])
        C, nt = cell.tangent(w["tol_cg"])
        nn_tot += nn
        nc_tot += nc
        nt_tot += nt
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev_ms = ev0.elapsed_time(ev1)
    prof = cell.profile_read()
    launches = cell.launches() - l0
    cell.close()
    del cell
    torch.cuda.empty_cache()
    bpv = fs_bytes_per_voxel(N)
    it = nc_tot + nt_tot  # CG iterations of the Newton and of the tangent solves
    solves = nn_tot + 9 * timed
    eff = {"fs_p1_cg_f32": it, "fs_p5_dot_f32": it, "fs_cg_update_f32": it,
           "fs_p1_cgf_f32": it, "fs_p5_cgf_f32": it, "fs_cg_rr_f32": it,
           "fs_p2_f32": it + solves + 9 * timed, "fs_p3_f32": it + solves + 9 * timed,
           "fs_p4_f32": it + solves + 9 * timed}
    kind, (kms, kn) = max(((k, v) for k, v in prof.items() if k in bpv), key=lambda kv: kv[1][0])
    hbm, peak_kind = measured_hbm()
    alg = eff[kind] * V * bpv[kind]
    achieved = alg / (kms * 1e-3) / 1e9
    fused = "fs_p1_cgf_f32" in prof
    it_kinds = (("fs_p1_cgf_f32", "fs_p2_f32", "fs_p3_f32", "fs_p4_f32", "fs_p5_cgf_f32", "fs_cg_rr_f32")
                if fused else
                ("fs_p1_cg_f32", "fs_p2_f32", "fs_p3_f32", "fs_p4_f32", "fs_p5_dot_f32", "fs_cg_update_f32"))
    iteration = None
    if all(k in prof and eff[k] for k in it_kinds):
        ims = sum(prof[k][0] / eff[k] for k in it_kinds)
        ib = sum(bpv[k] for k in it_kinds)
        ig = ib * V / (ims * 1e-3) / 1e9
        iteration = {"what": "one CG iteration, per field" + (" (update fused into P1/P5)" if fused else ""),
                     "ms_per_field_iter": round(ims, 4), "bytes_per_voxel": round(ib, 1),
                     "achieved": round(ig, 1), "peak": hbm, "unit": "GB/s", "frac": round(ig / hbm, 3)}
    return {
        "metric": f"CG-iter voxels/s at {N}^3, finite strain (FP32-inner mixed precision)",
        "value": V * it / (dev_ms * 1e-3), "unit": UNIT,
        "e2e_value": V * it / wall, "workload": f"fs_spheres{N}-stretch-shear",
        "step": "one load increment (Newton-CG) + 9x9 tangent",
        "increments_timed": timed, "newton_iters": nn_tot, "cg_iters": nc_tot, "tangent_cg_iters": nt_tot,
        "P": [float(v) for v in P.reshape(-1)], "ms": dev_ms, "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": measured_traffic(kind, N), "kernel": kind,
                     "peak_source": peak_kind, "bytes_per_launch": alg / max(eff[kind], 1),
                     "avg_launch_ms": kms / max(eff[kind], 1), "iteration": iteration},
        "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in sorted(
            prof.items(), key=lambda kv: -kv[1][0])},
    }


def cufft_matvec_line(N, iters=10):
    """Comparison line: q = G(C:p) with library FFTs (cuFFT through
    torch.fft rfftn/irfftn, FP32) and separate elementwise kernels for C:p
    and Ghat, on the same fields and compact tangent as the fused path.
    Returns ms per matvec (CUDA events, after warm-up)."""
    import torch
    dev = "cuda"
    g = torch.Generator(device=dev).manual_seed(0)
    p = torch.randn(6, N, N, N, device=dev, generator=g)
    K = torch.full((N, N, N), 0.833, device=dev)
    g2 = torch.full((N, N, N), 0.772, device=dev)
    w = 0.01 * torch.randn(5, N, N, N, device=dev, generator=g)
    k = torch.fft.fftfreq(N, d=1.0 / N, device=dev)
    k3 = torch.fft.rfftfreq(N, d=1.0 / N, device=dev)
    K1, K2, K3 = torch.meshgrid(k, k, k3, indexing="ij")
    q2 = K1 * K1 + K2 * K2 + K3 * K3
    inv = torch.where(q2 > 0, torch.rsqrt(torch.clamp(q2, min=1.0)), torch.zeros_like(q2))
    n = torch.stack([K1 * inv, K2 * inv, K3 * inv])
    scale = 1.0 / N ** 3

    def matvec(p):
        w0, w1, w23, w13, w12 = w
        w2 = -(w0 + w1)
        tr = p[0] + p[1] + p[2]
        m = tr / 3.0
        wp = w0 * p[0] + w1 * p[1] + w2 * p[2] + 2.0 * (w23 * p[3] + w13 * p[4] + w12 * p[5])
        s = torch.stack([K * tr + g2 * (p[0] - m) - wp * w0, K * tr + g2 * (p[1] - m) - wp * w1,
                         K * tr + g2 * (p[2] - m) - wp * w2, g2 * p[3] - wp * w23,
                         g2 * p[4] - wp * w13, g2 * p[5] - wp * w12])
        t = torch.fft.rfftn(s, dim=(1, 2, 3))
        v0 = n[0] * t[0] + n[1] * t[5] + n[2] * t[4]
        v1 = n[0] * t[5] + n[1] * t[1] + n[2] * t[3]
        v2 = n[0] * t[4] + n[1] * t[3] + n[2] * t[2]
        sn = n[0] * v0 + n[1] * v1 + n[2] * v2
        o = torch.stack([2 * n[0] * v0 - n[0] * n[0] * sn, 2 * n[1] * v1 - n[1] * n[1] * sn,
                         2 * n[2] * v2 - n[2] * n[2] * sn, n[1] * v2 + n[2] * v1 - n[1] * n[2] * sn,
                         n[0] * v2 + n[2] * v0 - n[0] * n[2] * sn, n[0] * v1 + n[1] * v0 - n[0] * n[1] * sn])
        q = torch.fft.irfftn(o * scale, s=(N, N, N), dim=(1, 2, 3)) * N ** 3
        return q, (p * q).sum()

    for _ in range(3):
        matvec(p)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        matvec(p)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    del p, K, g2, w, n, q2, inv, K1, K2, K3
    torch.cuda.empty_cache()
    return ms


# --------------------------------------------------------------- GPU leg
def fe2_pair_line(cell, w, start_inc, n_pairs=2):
    """The FE^2 call pair at the end of the load path: one increment of the
    path's size followed by the 6x6 tangent, `n_pairs` times, with the
    library's per-kernel events off (device-resident CG graphs). Device time
    by CUDA events; CG-iteration voxels/s as the headline counts them."""
    import torch
    N = w["N"]
    stream = cell.stream
    dE = w["dE"][0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    t0 = time.perf_counter()
    newton = cg = tcg = 0
    for _ in range(n_pairs):
        sig, nn, nc = cell.step(dE, w["tol_newton"], w["tol_cg"])
        C, nt = cell.tangent(w["tol_cg"])
        newton, cg, tcg = newton + nn, cg + nc, tcg + nt
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dev = e0.elapsed_time(e1) * 1e-3
    E11 = float(w["dE"][0][0] * (start_inc + n_pairs))
    return {"what": "increment + 6x6 tangent (the FE^2 Gauss-point call pair), CG graphs",
            "value": N ** 3 * (cg + tcg) / dev, "unit": UNIT, "ms_per_pair": 1e3 * dev / n_pairs,
            "e2e_ms_per_pair": 1e3 * wall / n_pairs, "pairs": n_pairs, "E11_end": E11,
            "newton_iters": newton, "cg_iters": cg, "tangent_cg_iters": tcg}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cores = os.cpu_count() or 1
    oracle = None
    fut_full = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # spawned before the first CUDA call; the full-grid oracle iteration
        # runs on one core while the GPU legs run
        oracle = oracle_pool(cores)
        fut_full = oracle.submit(oracle_job, args.N, 2 if args.N == 243 else 1, 1, args.N, 0)
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1601_05970_gb300 import build, fftg
    from paper_1601_05970_gb300 import inputs as I
    build.build()
    fftg.load()
    if args.finite_strain_only:
        if rank == 0:
            print(json.dumps(finite_strain_line(args.N)))
        return 0
    if args.projection_only:
        if rank == 0:
            print(json.dumps(projection_line(args.N, args.steps, args.warmup)))
        return 0

    N = args.N
    if args.steps > PATH_INCREMENTS:
        raise SystemExit(f"--steps {args.steps}: the load path has {PATH_INCREMENTS} increments")
    # schedules of the FP32 passes at every grid size the run uses, tuned
    # (or read from the schedule cache) before any handle is created
    tuned = {}
    if not args.no_tune:
        grids = [N] + ([] if args.no_extras or world > 1 else [15, 27, 45, 75, 135])
        for n in dict.fromkeys(grids):
            chosen, ms = fftg.autotune(n, cache=True)
            tuned[n] = {"chosen": chosen, "ms": ms}
    w = I.workload("spheres243" if N == 243 else "spheres135", seed=rank_seed(rank, 2 if N == 243 else 1))
    path = w["dE"]
    tol_nw, tol_cg = w["tol_newton"], w["tol_cg"]
    tangent = not args.no_tangent
    cell = fftg.Cell(N, w["phase"], w["mats"], precision=args.precision,
                     nrhs_tangent=6 if tangent else 0, cg_graph=0 if args.no_graph else 1)
    stream = cell.stream
    V = N ** 3

    def increment(k, acc):
        sig, nn, nc = cell.step(path[k], tol_nw, tol_cg)
        acc["newton"] += nn
        acc["cg"] += nc
        acc["sigma"] = sig

    # warm-up: the first increments of the path (and a tangent), then the
    # cell goes back to the undeformed state
    warm = dict(newton=0, cg=0)
    for k in range(min(args.warmup, PATH_INCREMENTS)):
        increment(k, warm)
    if tangent and args.warmup > 0:
        cell.tangent(tol_cg)
    cell.reset_state()
    cell.profile(True)
    cell.profile_reset()
    acc = dict(newton=0, cg=0, tangent_cg=0, tangent_calls=0)
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
        time.sleep(0.4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = cell.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()  # profiler range = the timed region (no effect without one)
    ev0.record(stream)
    t0 = time.perf_counter()
    for k in range(args.steps):
        increment(k, acc)
    if tangent:
        C, nt = cell.tangent(tol_cg)
        acc["tangent_cg"] += nt
        acc["tangent_calls"] += 1
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if not args.no_clocks else None
    launches = cell.launch_count() - launches0
    dev_ms = ev0.elapsed_time(ev1)
    wall_ms = 1e3 * (t1 - t0)
    prof = cell.profile_read()
    cell.profile(False)
    field_iters = acc["cg"] + acc["tangent_cg"]
    units = float(V) * field_iters
    if dist:
        dev_ms, wall_ms, units, launches = reduce_over_ranks(dist, dev_ms, wall_ms, units, launches,
                                                              "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline: the dominant kernel (largest device time in the timed
    # region), the matvec and the whole CG iteration
    sfx = "_f32" if args.precision == "mixed" else "_f64"
    hbm, peak_kind = measured_hbm()
    rf = cg_roofline(prof, N, field_iters, acc["newton"], acc["tangent_calls"], sfx, hbm)
    kind, (kms, kn) = max(prof.items(), key=lambda kv: kv[1][0])
    base = kind[:-len(sfx)] if kind.endswith(sfx) else None
    roof = None
    if base in rf["kernels"]:
        kr = rf["kernels"][base]
        per_launch = kr["bytes_per_voxel"] * V
        roof = {"bound": "hbm", "achieved": kr["GB/s"], "peak": hbm, "unit": "GB/s",
                "frac": kr["frac"], "traffic": measured_traffic(kind, N), "kernel": kind,
                "peak_source": peak_kind, "bytes_per_launch": per_launch, "avg_launch_ms": kr["ms"],
                "matvec": rf["matvec"], "iteration": rf["iteration"], "kernels": rf["kernels"]}
    E11_end = float(path[0][0] * args.steps) if N == 243 else None
    line = {
        "metric": METRIC, "value": units / (dev_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"spheres{N}-uniaxial" if N == 243 else f"spheres{N}-shear",
                   "N": N, "voxels": V, "precision": args.precision,
                   "hard_fraction": round(w["fraction"], 4), "seed": w["seed"],
                   "step": "one increment of the load path from the undeformed state (Newton-CG); "
                           + ("the 6x6 tangent after the last step is timed too" if tangent
                              else "no tangent"),
                   "path": f"{args.steps} of {PATH_INCREMENTS} increments, E11 to {E11_end}"
                   if N == 243 else f"{args.steps} of {PATH_INCREMENTS} shear increments",
                   "l2": "inputs larger than L2 (each FP32 field 344 MB)" if N == 243
                   else "inputs larger than L2 (each FP32 field 59 MB; spectra + fields > 129 MB)",
                   "parallelism": f"replicas x{world}",
                   "newton_iters": acc["newton"], "cg_iters": acc["cg"],
                   "tangent_cg_iters": acc["tangent_cg"],
                   "schedules": {str(n): t["chosen"] for n, t in tuned.items()}
                   if tuned else "defaults (--no-tune)"},
        "e2e": {"value": units / (wall_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 48, "d2h_bytes_per_step": 48 + (288 // args.steps if tangent else 0)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clocks,
        "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in sorted(
            prof.items(), key=lambda kv: -kv[1][0])},
    }
    if world == 1 and tangent and not args.no_extras and N == 243:
        line["config"]["fe2_pair"] = fe2_pair_line(cell, w, args.steps)
    if not args.no_extras and world == 1:
        cell.close()
        del cell
        torch.cuda.empty_cache()
        from paper_1601_05970_gb300 import serving
        fma64 = fftg.fma_rate("fp64")
        fma32 = fftg.fma_rate("fp32")
        pl = precision_lines(N, fma64=fma64)
        line["time_to_converged_stress"] = pl
        fp = pl["fp64"]
        line["config"]["fp64_plain"] = {
            "what": "plain FP64 path (FP64 CG, FFTs and residual), fresh cell, plastic increments "
                    "2-3 of the load path, no tangent; mixed on the same increments for comparison",
            "value": fp["cg_iter_voxels_per_s"], "unit": UNIT,
            "mixed_same_increments": pl["mixed"]["cg_iter_voxels_per_s"],
            "time_to_converged_stress_s": {"fp64": fp["seconds"], "mixed": pl["mixed"]["seconds"]},
            "speedup_mixed_over_fp64": pl.get("speedup_mixed_over_fp64"),
            "max_rel_diff_sigma": pl["fp64"].get("max_rel_diff_sigma_vs_mixed"),
            "iteration_ms": fp["iteration_ms"], "roofline": fp.get("roofline"),
            "fma_tflops": {"fp64": fma64, "fp32": fma32}}
        fused = rf["matvec"]["ms_per_field_iter"] if rf["matvec"] else None
        line["cufft_line"] = {"matvec_ms": cufft_matvec_line(N), "fused_matvec_ms": fused,
                              "what": "q = G(C:p) at N^3 FP32: cuFFT rfftn/irfftn via torch.fft with "
                                      "separate elementwise C:p and Ghat kernels, vs the fused passes "
                                      "P1-P5 per CG field-iteration in the timed region"}
        line["basic_scheme_vs_cg"] = basic_scheme_line()
        line["finite_strain"] = finite_strain_line()
        rves = serving.batched_workload()
        line["batched"] = serving.run_batched(rves, graph=True)
        line["batched_threads"] = serving.run_batched(rves, graph=False)
        line["config"]["batched"] = {k: line["batched"][k] for k in ("rves", "increments", "solves_per_s",
                                                                     "mode", "graph_launches")}
        line["config"]["batched"]["threads_solves_per_s"] = line["batched_threads"]["solves_per_s"]
        rates = [float(r) for r in args.serve_rates.split(",")]
        sv = [serving.run(r, args.serve_seconds) for r in rates]
        line["serving"] = sv
        line["config"]["serving"] = [{k: s.get(k) for k in ("rate", "solves_per_s", "p50_ms", "p99_ms",
                                                            "completed", "requests", "backlog")}
                                     for s in sv]
    else:
        cell.close()
    if oracle is not None:
        single = oracle.submit(oracle_job, N, w["seed"], 2, 63, 0).result()
        st_rate = single[0] / (single[2] - single[1])
        allc = oracle_all_cores(oracle, max(1, cores - 1), N, w["seed"])
        per_n = oracle_per_n(oracle)
        units_full, t0f, t1f = fut_full.result()
        oracle.shutdown()
        per_n[str(N)] = units_full / (t1f - t0f)
        line["cpu_baseline"] = {
            "value": allc, "unit": UNIT, "cores": max(1, cores - 1), "kind": "oracle",
            "sample": (f"FP64 numpy oracle, 2 CG iterations (G C p on full 3x3 tensors and the vector "
                       f"updates) on each of {max(1, cores - 1)} 63^3 blocks of the {N}^3 workload at "
                       f"once, one single-threaded process per core (host nproc = {cores})"),
            "single_thread": {"value": st_rate, "sample": f"one 63^3 block of the {N}^3 workload, "
                                                          "2 CG iterations, 1 thread"},
            "per_N_single_thread": per_n,
            "fixed_20_iterations_full_grid_s": {
                "value": 20 * (t1f - t0f), "extrapolated": True,
                "what": f"one oracle CG iteration on the whole {N}^3 cell (1 thread) x 20"},
        }
    if tuned:
        line["autotune"] = {str(n): t for n, t in tuned.items()}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
