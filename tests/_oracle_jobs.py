"""Oracle reference computations of the full-size parity tests, run in
worker processes (spawned, so no CUDA state is inherited) while the GPU side
of the tests runs. Each job builds its inputs from the seeded generators,
runs the FP64 oracle and saves the inputs and expected values to an .npz
file; nothing here touches the CUDA path.
"""
import os

import numpy as np

E_PLASTIC = np.array([0.00075, -0.000375, 0.0001875, 0.000375, -0.00075, 0.001125])


def matvec_case(N, outdir):
    """Oracle G (C : p) on the N^3 sphere workload with a random fluctuation
    that makes part of the voxels yield; p is FP32-representable. Also the
    oracle's tangent on a fixed sample of voxels, applied to a random
    direction."""
    from oracle import fftg_oracle as O
    from paper_1601_05970_gb300 import inputs as I
    w = I.workload(f"spheres{N}")
    rng = np.random.default_rng(100 + N)
    eps = 0.0015 * rng.standard_normal((6, N, N, N))
    st = O.State(N, w["phase"], w["mats"])
    res = st.constitutive(O.to_tensor(E_PLASTIC), O.to_tensor(eps))
    p = rng.standard_normal((6, N, N, N)).astype(np.float32).astype(np.float64)
    pt = O.to_tensor(p)
    q = O.matvec(O.Tangent(res), pt)
    srng = np.random.default_rng(7)
    idx = np.sort(srng.choice(N ** 3, size=20000, replace=False))
    Cs = O.j2_tangent(res, idx)
    ps = srng.standard_normal((6, idx.size))
    cs = O.to_comps(np.einsum("ijlmv,lmv->ijv", Cs, O.to_tensor(ps)))
    path = os.path.join(outdir, f"matvec_{N}.npz")
    np.savez(path, eps=eps, sigma=O.to_comps(res.sigma), p=p, q=O.to_comps(q), pq=O.inner(pt, q),
             plastic=res.plastic.mean(), idx=idx, ps=ps, cps=cs, cscale=np.abs(Cs).max(),
             plastic_sample=res.plastic.reshape(-1)[idx].mean())
    return path


def fixed_solve_case(N, E0, dE, n_inc, fixed_cg, fixed_newton, outdir):
    """Increments of Algorithm 1 in the fixed-iteration mode on the N^3
    shear workload, from the committed state (E0, eps* = 0, no history)."""
    from oracle import fftg_oracle as O
    from paper_1601_05970_gb300 import inputs as I
    w = I.workload(f"spheres{N}")
    st = O.State(N, w["phase"], w["mats"], E=O.to_tensor(np.asarray(E0, dtype=np.float64)))
    sig, counts, eps = [], [], []
    for _ in range(n_inc):
        r = O.solve_increment(st, dE, 1e-5, 1e-8, fixed_cg=fixed_cg, fixed_newton=fixed_newton)
        sig.append(r.sigma)
        counts.append((r.newton_iters, r.cg_iters))
        eps.append(O.to_comps(st.eps_star) + O.to_comps(st.E)[:, None, None, None])
    path = os.path.join(outdir, f"solve_{N}.npz")
    np.savez(path, sigma=np.array(sig), counts=np.array(counts), eps=np.array(eps), epbar=st.epbar)
    return path
