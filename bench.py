#!/usr/bin/env python
"""Benchmark of the FFT-Galerkin Newton-CG solver on one or more GB300s.

Workload: the 243^3 periodic cell with random hard spheres (radii 3-8,
hard fraction 0.2), J2 with linear hardening, uniaxial strain E11 ramped
in increments of 0.0015, mixed precision (FP32 inner CG, FP64 return
mapping, residual and homogenisation). One step = one load increment
(Newton-CG to 1e-5 / CG 1e-8, floor 1e-6 in FP32) followed by the 6x6
macroscopic tangent (six right-hand sides in one batched CG): the call pair
an FE^2 macro solver makes per Gauss point. The warm-up increments take the
cell past first yield, so the timed increments are plastic.

Metric: CG-iteration voxels/s = N^3 x (CG iterations of the Newton solves +
CG iterations of the six tangent solves) / time.

With --gpus N under torchrun each rank solves its own cell (own seed): the
path shards by cell with no data exchange (replicas; weak scaling).
`--impl reference` times the FP64 numpy oracle on the host instead.
"""
import os

# the oracle legs must use one host thread (counted as `cores`)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG-iter voxels/s at 243^3 (FP32-inner mixed precision)"
UNIT = "voxel-iterations/s"

# Algorithmic bytes per voxel and per field of each kernel kind (what the
# kernel must read and write given its interface; FP32 fields are 24 B per
# voxel, the half spectrum 6 x (H/N) x 8 B, the compact tangent 28 B).
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
        "p1_tanrhs_f32": 28 + s32,
        "p5_rhs_f32_to_f32": s32 + 24,
        "p1_plain_f64": 48 + s64, "p2_f64": 2 * s64, "p3_f64": 2 * s64, "p4_f64": 2 * s64,
        "p5_rhs_f64_to_f32": s64 + 24,
    }


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the dominant kernels from one ncu capture each (profiles/traffic_cg_kernels_
# spheres243.md, profiles/traffic_fs_cg_kernels_spheres243.md), valid while
# the kernel sources have the digest they had then (SHA-256 prefix of the
# files listed).
KERNEL_FILES = ("common.cuh", "fft_core.cuh", "passes.cuh")
FS_KERNEL_FILES = KERNEL_FILES + ("fs_passes.cuh",)
TRAFFIC = {"p1_cg_f32": {"N": 243, "bytes": 2418.1e6, "digest": "7933c1ea13abe27e", "files": KERNEL_FILES},
           "fs_p1_cg_f32": {"N": 243, "bytes": 3579.6e6, "digest": "23608171e96a0ffe", "files": FS_KERNEL_FILES}}


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
    ap.add_argument("--steps", type=int, default=5)
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
    ap.add_argument("--finite-strain-only", action="store_true",
                    help="run only the finite-strain line (mixed, --N 243 or 135) and print it")
    ap.add_argument("--serve-rate", type=float, default=100.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
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
def oracle_sample(N_full, seed, n_iters, sub=81):
    """Time `n_iters` oracle CG iterations on the sub x sub x sub corner of the
    same microstructure (periodic closure), after one constitutive
    evaluation at the macroscopic strain the timed GPU increments start from
    (E11 = 0.0045, zero history, eps* = 0). Returns (voxel-iterations/s, desc)."""
    from oracle import fftg_oracle as O
    from paper_1601_05970_gb300 import inputs as I
    w = I.workload("spheres243" if N_full == 243 else "spheres135", seed=seed)
    ph = np.ascontiguousarray(w["phase"][:sub, :sub, :sub])
    st = O.State(sub, ph, w["mats"])
    E = O.to_tensor(np.array([0.0045, 0, 0, 0, 0, 0]))
    res = st.constitutive(E, np.zeros((3, 3, sub, sub, sub)))
    tan = O.Tangent(res)
    b = -O.project(res.sigma)
    t0 = time.perf_counter()
    O.cg(lambda p: O.matvec(tan, p), b, 1e-30, fixed_iters=n_iters)
    dt = time.perf_counter() - t0
    desc = (f"FP64 numpy oracle, {n_iters} CG iterations (G C p on full 3x3 tensors) on the "
            f"{sub}^3 corner of the {N_full}^3 microstructure (seed {seed}), 1 host thread")
    return sub ** 3 * n_iters / dt, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    for k in range(args.warmup + args.steps):
        v, desc = oracle_sample(args.N, 2, 1)
        if k >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    ms = 1e3 * (81 ** 3) / value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"spheres{args.N}-uniaxial (oracle sample)", "N": args.N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- ranks
def rank_seed(rank):
    """Each rank solves its own cell: the microstructure seed of rank r."""
    return 2 + 1000 * rank


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
def time_to_converged_stress(N, precisions=("mixed", "fp64"), n_inc=4, timed_from=2):
    """Wall time of increments timed_from.. of the uniaxial path at N^3 for
    each precision, on fresh cells (no tangent): the first increments are
    elastic, the timed ones plastic."""
    import torch
    from paper_1601_05970_gb300 import fftg
    from paper_1601_05970_gb300 import inputs as I
    w = I.workload("spheres243" if N == 243 else "spheres135")
    out = {}
    sig_ref = None
    for prec in precisions:
        cell = fftg.Cell(N, w["phase"], w["mats"], precision=prec, nrhs_tangent=0)
        t_tot, iters = 0.0, []
        for k in range(n_inc):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sig, nn, nc = cell.step(w["dE"][k], w["tol_newton"], w["tol_cg"])
            torch.cuda.synchronize()
            if k >= timed_from:
                t_tot += time.perf_counter() - t0
                iters.append((nn, nc))
        out[prec] = dict(seconds=t_tot, increments=n_inc - timed_from, newton_cg=iters,
                         sigma=[float(v) for v in sig])
        if sig_ref is None:
            sig_ref = sig
        else:
            out[prec]["max_rel_diff_sigma_vs_" + precisions[0]] = float(
                np.abs(sig - sig_ref).max() / np.abs(sig_ref).max())
        cell.close()
        del cell
        torch.cuda.empty_cache()
    if "mixed" in out and "fp64" in out:
        out["speedup_mixed_over_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


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
            "fs_p5_dot_f32": s32 + 36 + 36, "fs_cg_update_f32": 3 * 36}


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
           "fs_p2_f32": it + solves + 9 * timed, "fs_p3_f32": it + solves + 9 * timed,
           "fs_p4_f32": it + solves + 9 * timed}
    kind, (kms, kn) = max(((k, v) for k, v in prof.items() if k in bpv), key=lambda kv: kv[1][0])
    hbm, peak_kind = measured_hbm()
    alg = eff[kind] * V * bpv[kind]
    achieved = alg / (kms * 1e-3) / 1e9
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
                     "avg_launch_ms": kms / max(eff[kind], 1)},
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
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
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

    N = args.N
    w = I.workload("spheres243" if N == 243 else "spheres135", seed=rank_seed(rank))
    dE = np.array([0.0015, 0, 0, 0, 0, 0]) if N == 243 else np.array([0, 0, 0, 0, 0, 0.001])
    tol_nw, tol_cg = w["tol_newton"], w["tol_cg"]
    cell = fftg.Cell(N, w["phase"], w["mats"], precision=args.precision,
                     nrhs_tangent=0 if args.no_tangent else 6,
                     cg_graph=0 if args.no_graph else 1)
    stream = cell.stream
    V = N ** 3

    def one_step(acc):
        sig, nn, nc = cell.step(dE, tol_nw, tol_cg)
        acc["newton"] += nn
        acc["cg"] += nc
        if not args.no_tangent:
            C, nt = cell.tangent(tol_cg)
            acc["tangent_cg"] += nt
            acc["tangent_calls"] += 1
        acc["sigma"] = sig

    warm = dict(newton=0, cg=0, tangent_cg=0, tangent_calls=0)
    for _ in range(args.warmup):
        one_step(warm)
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
    for _ in range(args.steps):
        one_step(acc)
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
    field_iters = acc["cg"] + acc["tangent_cg"]
    units = float(V) * field_iters
    if dist:
        dev_ms, wall_ms, units, launches = reduce_over_ranks(dist, dev_ms, wall_ms, units, launches,
                                                              "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (largest device time in the timed region)
    bpv = bytes_per_voxel(N)
    kind, (kms, kn) = max(prof.items(), key=lambda kv: kv[1][0])
    # effective field-launches of the CG kernels = CG field-iterations
    # (chunked launches past convergence return at entry and do no work)
    eff = {"p1_cg_f32": field_iters, "p5_dot_f32": field_iters, "cg_update_f32": field_iters,
           "p2_f32": field_iters + 6 * acc["tangent_calls"],
           "p3_f32": field_iters + 6 * acc["tangent_calls"],
           "p4_f32": field_iters + 6 * acc["tangent_calls"]}
    hbm, peak_kind = measured_hbm()
    roof = None
    if kind in bpv and kind in eff:
        alg_bytes = eff[kind] * V * bpv[kind]
        achieved = alg_bytes / (kms * 1e-3) / 1e9
        per_launch = alg_bytes / max(eff[kind], 1)
        traffic = measured_traffic(kind, N)
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "kernel": kind,
                "peak_source": peak_kind, "bytes_per_launch": per_launch,
                "avg_launch_ms": kms / max(eff[kind], 1)}
    line = {
        "metric": METRIC, "value": units / (dev_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"spheres{N}-uniaxial", "N": N, "voxels": V,
                   "precision": args.precision, "hard_fraction": round(w["fraction"], 4),
                   "seed": w["seed"], "step": "one load increment (Newton-CG) + 6x6 tangent"
                   if not args.no_tangent else "one load increment (Newton-CG)",
                   "l2": "inputs larger than L2 (each FP32 field 344 MB)" if N == 243
                   else "inputs larger than L2 (each FP32 field 59 MB; spectra + fields > 129 MB)",
                   "parallelism": f"replicas x{world}",
                   "newton_iters": acc["newton"], "cg_iters": acc["cg"],
                   "tangent_cg_iters": acc["tangent_cg"]},
        "e2e": {"value": units / (wall_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 48,
                "d2h_bytes_per_step": 48 + (288 if not args.no_tangent else 0)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clocks,
        "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in sorted(
            prof.items(), key=lambda kv: -kv[1][0])},
    }
    if not args.no_cpu_baseline and world == 1:
        v, desc = oracle_sample(N, w["seed"], 3)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    if not args.no_extras and world == 1:
        cell.close()
        del cell
        torch.cuda.empty_cache()
        from paper_1601_05970_gb300 import serving
        fused = sum(line["kernels"].get(k, {"ms": 0.0})["ms"] for k in
                    ("p1_cg_f32", "p2_f32", "p3_f32", "p4_f32", "p5_dot_f32")) / max(field_iters, 1)
        line["cufft_line"] = {"matvec_ms": cufft_matvec_line(N), "fused_matvec_ms": fused,
                              "what": "q = G(C:p) at N^3 FP32: cuFFT rfftn/irfftn via torch.fft with "
                                      "separate elementwise C:p and Ghat kernels, vs the fused passes "
                                      "P1-P5 per CG field-iteration in the timed region"}
        line["time_to_converged_stress"] = time_to_converged_stress(N)
        line["basic_scheme_vs_cg"] = basic_scheme_line()
        line["finite_strain"] = finite_strain_line()
        rves = serving.batched_workload()
        line["batched"] = serving.run_batched(rves)
        line["serving"] = serving.run(args.serve_rate, args.serve_seconds, budget_gb=48.0)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
