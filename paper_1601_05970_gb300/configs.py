"""Full runs of the five workload configurations, printed as one JSON line.

    python -m paper_1601_05970_gb300.configs [--skip 4,5] [--only 6]

1. 15^3 laminate, FP64 and mixed, shear to 0.02 in 10 increments: the
   homogenised shear stress against the closed form of the laminate (both
   phases in pure shear with equal elasticity, so only eps_12 differs
   between them; Section 4.2 with linear hardening).
2. 135^3 spheres (hard fraction 0.3), shear to 0.02 in 20 increments, FP64
   against mixed precision: wall time, iteration counts, stress difference.
3. 243^3 spheres (hard fraction 0.2), uniaxial strain to 0.03 in 20
   increments, then the 6x6 macroscopic tangent.
4. 256 RVEs of mixed sizes, 5 increments each (serving.run_batched).
5. The serving loop at 50, 100, 200 and 500 requests/s (serving.run).
6. Finite strain: the 45^3 laminate (FP64 and mixed) at 30 % deformation
   against its two-layer closed form, then the 243^3 spheres stretch-shear
   path (5 increments, mixed) and the 9x9 macroscopic tangent.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def _laminate_shear_closed_form(E12, G, f_h, hard, soft):
    """Sigma_12 of the laminate: tau_h(g_h) = tau_s(g_s), f_h g_h + (1-f_h) g_s
    = 2 E12, with tau(g) = G g below sigma_0/sqrt3 and
    (sigma_0/sqrt3 + H g/3)/(1 + H/(3G)) above (monotone pure shear)."""
    from scipy.optimize import brentq

    def tau(g, sy, H):
        return G * g if G * g <= sy / math.sqrt(3) else (sy / math.sqrt(3) + H * g / 3) / (1 + H / (3 * G))

    F = lambda gh: tau(gh, hard.sigma_y, hard.H) - tau((2 * E12 - f_h * gh) / (1 - f_h), soft.sigma_y, soft.H)
    gh = brentq(F, 0.0, 2 * E12 / f_h, xtol=1e-300, rtol=1e-15)
    return tau(gh, hard.sigma_y, hard.H)


def config1():
    from . import fftg, inputs as I
    w = I.workload("laminate15")
    soft, hard = I.TWO_PHASE
    rows = []
    for prec in ("fp64", "mixed"):
        cell = fftg.Cell(15, w["phase"], w["mats"], precision=prec)
        E12, errs, nn_t, nc_t = 0.0, [], 0, 0
        for dE in w["dE"]:
            sig, nn, nc = cell.step(dE, w["tol_newton"], w["tol_cg"])
            nn_t += nn
            nc_t += nc
            E12 += dE[5]
            S12 = _laminate_shear_closed_form(E12, soft.G, 5 / 15, hard, soft)
            errs.append(abs(sig[5] - S12) / S12)
        rows.append(dict(precision=prec, max_rel_err_sigma12=max(errs), newton=nn_t, cg=nc_t))
        cell.close()
    return rows


def _timed_path(cell, dEs, tol_newton, tol_cg):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nn_t = nc_t = 0
    for dE in dEs:
        sig, nn, nc = cell.step(dE, tol_newton, tol_cg)
        nn_t += nn
        nc_t += nc
    torch.cuda.synchronize()
    return time.perf_counter() - t0, nn_t, nc_t, sig


def config2():
    import torch
    from . import fftg, inputs as I
    w = I.workload("spheres135")
    res = {}
    for prec in ("fp64", "mixed"):
        cell = fftg.Cell(135, w["phase"], w["mats"], precision=prec, nrhs_tangent=0)
        t, nn, nc, sig = _timed_path(cell, w["dE"], w["tol_newton"], w["tol_cg"])
        res[prec] = dict(seconds=t, newton=nn, cg=nc, sigma=[float(v) for v in sig])
        cell.close()
        torch.cuda.empty_cache()
    s64, s32 = np.array(res["fp64"]["sigma"]), np.array(res["mixed"]["sigma"])
    res["max_rel_diff_sigma"] = float(np.abs(s64 - s32).max() / np.abs(s64).max())
    res["speedup_mixed"] = res["fp64"]["seconds"] / res["mixed"]["seconds"]
    return res


def config3():
    import torch
    from . import fftg, inputs as I
    w = I.workload("spheres243")
    cell = fftg.Cell(243, w["phase"], w["mats"], precision="mixed")
    t, nn, nc, sig = _timed_path(cell, w["dE"], w["tol_newton"], w["tol_cg"])
    t1 = time.perf_counter()
    C, tc = cell.tangent(w["tol_cg"])
    torch.cuda.synchronize()
    out = dict(path_seconds=t, newton=nn, cg=nc, sigma=[float(v) for v in sig],
               tangent_seconds=time.perf_counter() - t1, tangent_cg=tc,
               tangent=np.asarray(C).tolist(),
               tangent_asymmetry=float(np.abs(C - C.T).max() / np.abs(C).max()))
    cell.close()
    return out


def _svk_P(F, lam, mu):
    """First Piola-Kirchhoff stress of St. Venant-Kirchhoff, P = F S."""
    E = 0.5 * (F.T @ F - np.eye(3))
    return F @ (lam * np.trace(E) * np.eye(3) + 2.0 * mu * E)


def _laminate_fs_closed_form(Fbar, f_h, hard, soft):
    """Mean P of two layers normal to e1: F_k = Fbar + a_k (x) e1 with
    f_h a_h + (1 - f_h) a_s = 0 and P e1 continuous across the interface."""
    from scipy.optimize import fsolve

    def P_of(a, m):
        return _svk_P(Fbar + np.outer(a, [1.0, 0.0, 0.0]), m.lam, m.mu)

    def resid(a_h):
        return (P_of(a_h, hard) - P_of(-f_h / (1.0 - f_h) * a_h, soft))[:, 0]

    a_h = fsolve(resid, np.zeros(3), xtol=1e-15)
    return f_h * P_of(a_h, hard) + (1.0 - f_h) * P_of(-f_h / (1.0 - f_h) * a_h, soft)


def config6():
    import torch
    from . import fftg, inputs as I
    out = {}
    N, n_h = 45, 17
    dF = 0.3 * np.array([[0.5, 0.4, -0.2], [0.3, -0.2, 0.25], [0.1, 0.35, 0.2]])
    P_ref = _laminate_fs_closed_form(np.eye(3) + dF, n_h / N, I.SVK_HARD, I.SVK_SOFT)
    for prec, tn, tc in (("fp64", 1e-10, 1e-12), ("mixed", 1e-8, 1e-8)):
        cell = fftg.FsCell(N, I.laminate(N, n_h, axis=0), I.SVK_TWO_PHASE, precision=prec)
        P, nn, nc = cell.step(dF, tn, tc)
        out[f"laminate45_{prec}"] = dict(max_rel_err_P=float(np.abs(P - P_ref).max() / np.abs(P_ref).max()),
                                         newton=nn, cg=nc)
        cell.close()
    w = I.workload("fs_spheres243")
    cell = fftg.FsCell(243, w["phase"], w["mats"], precision="mixed")
    t, nn, nc, P = _timed_path(cell, w["dF"][:5], w["tol_newton"], w["tol_cg"])
    t1 = time.perf_counter()
    C, ntc = cell.tangent(w["tol_cg"])
    torch.cuda.synchronize()
    out["spheres243"] = dict(path_seconds=t, increments=5, newton=nn, cg=nc,
                             P=np.asarray(P).reshape(-1).tolist(),
                             tangent_seconds=time.perf_counter() - t1, tangent_cg=ntc,
                             tangent_asymmetry=float(np.abs(C - C.T).max() / np.abs(C).max()))
    cell.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--skip", default="", help="comma-separated configurations to leave out")
    ap.add_argument("--only", default="", help="comma-separated configurations to run (default: all)")
    args = ap.parse_args(argv)
    skip = {int(s) for s in args.skip.split(",") if s}
    if args.only:
        skip = set(range(1, 7)) - {int(s) for s in args.only.split(",") if s}
    out = {}
    if 1 not in skip:
        out["config1"] = config1()
    if 2 not in skip:
        out["config2"] = config2()
    if 3 not in skip:
        out["config3"] = config3()
    if 4 not in skip or 5 not in skip:
        from . import serving
        if 4 not in skip:
            out["config4"] = serving.run_batched(serving.batched_workload())
        if 5 not in skip:
            out["config5"] = [serving.run(rate, 10.0) for rate in (50.0, 100.0, 200.0, 500.0)]
    if 6 not in skip:
        out["config6"] = config6()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
