"""Thin Python binding of the fftg C-ABI (include/fftg.h, include/fftg_fs.h).

Argument marshalling only: every step of the solver runs in the CUDA
kernels of libfftg.so. The functions keep the C names; `Cell` wraps a
small-strain handle with PyTorch-allocated device memory and the current
torch stream, `FsCell` a finite-strain handle.
There is no CPU fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfftg.so")

FFTG_OK = 0
FFTG_EINVAL = -1
FFTG_ENOMEM = -2
FFTG_ENOCONV_NEWTON = -3
FFTG_ENOCONV_CG = -4
FFTG_ENAN = -5
FFTG_ECUDA = -6
FFTG_ESTATE = -7
FFTG_FP64 = 0
FFTG_MIXED = 1
FFTG_DD = 2
FFTG_SOLVER_CG = 0
FFTG_SOLVER_RICHARDSON = 1
FFTG_MODEL_J2, FFTG_MODEL_NLELASTIC, FFTG_MODEL_VISCO = 0, 1, 2
FFTG_FIELD_STRAIN = 0
FFTG_FIELD_STRESS = 1
FFTG_FIELD_EPBAR = 2
FFTG_FIELD_EPS_P = 3
FFTG_FIELD_TANGENT = 4
FFTG_MAX_NEWTON_LOG = 64
FFTG_FS_FIELD_DEFGRAD = 0
FFTG_FS_FIELD_STRESS = 1

ERRORS = {
    FFTG_EINVAL: "invalid argument",
    FFTG_ENOMEM: "out of device memory / workspace too small",
    FFTG_ENOCONV_NEWTON: "Newton did not converge",
    FFTG_ENOCONV_CG: "CG did not converge",
    FFTG_ENAN: "NaN or Inf in a residual",
    FFTG_ECUDA: "CUDA error",
    FFTG_ESTATE: "call out of order",
}


class FftgError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {ERRORS.get(code, 'error')} ({code})")
        self.code = code


class fftg_phase(C.Structure):
    _fields_ = [("K", C.c_double), ("G", C.c_double), ("sigma_y", C.c_double), ("H", C.c_double),
                ("n", C.c_double), ("eps0", C.c_double), ("t0", C.c_double), ("model", C.c_int)]


class fftg_svk_phase(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("mu", C.c_double)]


def svk_array(mats):
    """fftg_svk_phase[] from (lambda, mu) pairs or objects with as_tuple()."""
    arr = (fftg_svk_phase * len(mats))()
    for i, m in enumerate(mats):
        lam, mu = m.as_tuple() if hasattr(m, "as_tuple") else m
        arr[i].lambda_, arr[i].mu = float(lam), float(mu)
    return arr


def phase_array(mats):
    """fftg_phase[] from materials: objects with as_tuple() (inputs.Phase,
    NonlinearElastic, ViscoPlastic) or tuples (K, G, sigma_y, H[, n]) of a
    J2 phase, n = 1 by default."""
    from . import inputs
    rows = []
    for m in mats:
        t = inputs.material_tuple(m)
        rows.append(fftg_phase(*t[:7], int(t[7])))
    return (fftg_phase * len(rows))(*rows)


class fftg_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_newton", C.c_int), ("max_cg", C.c_int),
                ("cg_inner_floor", C.c_double), ("fixed_cg", C.c_int), ("fixed_newton", C.c_int),
                ("stream", C.c_void_p), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
                ("nrhs_tangent", C.c_int), ("cg_graph", C.c_int), ("dt", C.c_double),
                ("solver", C.c_int)]


class fftg_result(C.Structure):
    _fields_ = [("request_id", C.c_longlong), ("session_id", C.c_longlong), ("status", C.c_int),
                ("newton_iters", C.c_int), ("cg_iters", C.c_int), ("sigma", C.c_double * 6),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double)]


class fftg_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("cg_iters", C.c_int),
                ("cg_per_newton", C.c_int * FFTG_MAX_NEWTON_LOG),
                ("newton_norm", C.c_double * FFTG_MAX_NEWTON_LOG),
                ("residual", C.c_double * FFTG_MAX_NEWTON_LOG),
                ("cg_relres", C.c_double * FFTG_MAX_NEWTON_LOG),
                ("cg_status", C.c_int * FFTG_MAX_NEWTON_LOG)]


# every symbol include/fftg.h declares, with its ctypes signature
_D6 = C.POINTER(C.c_double)
SIGNATURES = {
    "fftg_default_options": (None, [C.POINTER(fftg_options)]),
    "fftg_version": (C.c_char_p, []),
    "fftg_workspace_size": (C.c_int, [C.c_int, C.POINTER(fftg_options), C.POINTER(C.c_size_t)]),
    "fftg_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_uint8), C.c_int,
                              C.POINTER(fftg_phase), C.POINTER(fftg_options)]),
    "fftg_step": (C.c_int, [C.c_void_p, _D6, C.c_double, C.c_double, _D6,
                            C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fftg_last_stats": (C.c_int, [C.c_void_p, C.POINTER(fftg_stats)]),
    "fftg_tangent": (C.c_int, [C.c_void_p, C.c_double, _D6, C.POINTER(C.c_int)]),
    "fftg_state_bytes": (C.c_size_t, [C.c_void_p]),
    "fftg_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fftg_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fftg_get_field": (C.c_int, [C.c_void_p, C.c_int, _D6]),
    "fftg_destroy": (None, [C.c_void_p]),
    "fftg_op_project": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "fftg_op_constitutive": (C.c_int, [C.c_void_p, _D6, C.c_void_p, C.c_void_p]),
    "fftg_op_matvec": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, _D6]),
    "fftg_profile_kinds": (C.c_int, []),
    "fftg_profile_name": (C.c_char_p, [C.c_int]),
    "fftg_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "fftg_profile_reset": (C.c_int, [C.c_void_p]),
    "fftg_profile_read": (C.c_int, [C.c_void_p, C.c_int, _D6, C.POINTER(C.c_longlong)]),
    "fftg_launch_count": (C.c_longlong, [C.c_void_p]),
    "fftg_reset_state": (C.c_int, [C.c_void_p]),
    "fftg_probe_fma_rate": (C.c_int, [C.c_int, C.c_int, C.c_void_p, _D6]),
    "fftg_schedule_set": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "fftg_schedule_get": (C.c_int, [C.c_int, C.c_int]),
    "fftg_schedule_describe": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "fftg_autotune": (C.c_int, [C.c_int, C.c_int, C.c_void_p, _D6, C.POINTER(C.c_int)]),
    "fftg_workspace_size_batch": (C.c_int, [C.c_int, C.c_int, C.POINTER(fftg_options),
                                            C.POINTER(C.c_size_t)]),
    "fftg_create_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_uint8),
                                    C.c_int, C.POINTER(fftg_phase), C.POINTER(fftg_options)]),
    "fftg_batch_size": (C.c_int, [C.c_void_p]),
    "fftg_select_cell": (C.c_int, [C.c_void_p, C.c_int]),
    "fftg_batch_step": (C.c_int, [C.c_void_p, _D6, C.c_double, C.c_double, _D6,
                                  C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fftg_group_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int]),
    "fftg_group_step": (C.c_int, [C.c_void_p, _D6, C.POINTER(C.c_int), C.c_double, C.c_double, _D6,
                                  C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fftg_group_launch_count": (C.c_longlong, [C.c_void_p]),
    "fftg_group_destroy": (None, [C.c_void_p]),
    "fftg_server_clock": (C.c_double, []),
    "fftg_server_start": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int,
                                    C.POINTER(fftg_phase), C.POINTER(fftg_options), C.c_double,
                                    C.c_double]),
    "fftg_server_submit": (C.c_int, [C.c_void_p, C.c_longlong, C.c_longlong, C.POINTER(C.c_uint8),
                                     _D6]),
    "fftg_server_poll": (C.c_int, [C.c_void_p, C.POINTER(fftg_result), C.c_int, C.POINTER(C.c_int),
                                   C.c_double]),
    "fftg_server_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_longlong), C.POINTER(C.c_int), _D6]),
    "fftg_server_stop": (C.c_int, [C.c_void_p]),
    "fftg_server_cancel_pending": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "fftg_constitutive_noalloc": (C.c_int, [C.c_int, _D6, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_int, C.POINTER(fftg_phase), C.c_int,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, _D6,
                                            C.c_void_p]),
    "fftg_fs_workspace_size": (C.c_int, [C.c_int, C.POINTER(fftg_options), C.POINTER(C.c_size_t)]),
    "fftg_fs_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_uint8), C.c_int,
                                 C.POINTER(fftg_svk_phase), C.POINTER(fftg_options)]),
    "fftg_fs_step": (C.c_int, [C.c_void_p, _D6, C.c_double, C.c_double, _D6,
                               C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fftg_fs_last_stats": (C.c_int, [C.c_void_p, C.POINTER(fftg_stats)]),
    "fftg_fs_tangent": (C.c_int, [C.c_void_p, C.c_double, _D6, C.POINTER(C.c_int)]),
    "fftg_fs_get_field": (C.c_int, [C.c_void_p, C.c_int, _D6]),
    "fftg_fs_state_bytes": (C.c_size_t, [C.c_void_p]),
    "fftg_fs_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fftg_fs_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fftg_fs_op_project": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "fftg_fs_op_matvec": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, _D6]),
    "fftg_fs_profile_kinds": (C.c_int, []),
    "fftg_fs_profile_name": (C.c_char_p, [C.c_int]),
    "fftg_fs_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "fftg_fs_profile_read": (C.c_int, [C.c_void_p, C.c_int, _D6, C.POINTER(C.c_longlong)]),
    "fftg_fs_launch_count": (C.c_longlong, [C.c_void_p]),
    "fftg_fs_destroy": (None, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfftg.so (raises OSError if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libfftg.so not built at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code, where):
    if code != FFTG_OK:
        raise FftgError(code, where)


def _dptr(a):
    return a.ctypes.data_as(_D6)


def default_options() -> fftg_options:
    o = fftg_options()
    load().fftg_default_options(C.byref(o))
    return o


def workspace_size(N: int, opt: fftg_options) -> int:
    b = C.c_size_t(0)
    check(load().fftg_workspace_size(N, C.byref(opt), C.byref(b)), "fftg_workspace_size")
    return b.value


class Cell:
    """A handle of one or more periodic cells whose device memory comes from
    PyTorch.

    phase: uint8 [N, N, N] (x1 slowest), or [ncells, N, N, N] for a batch;
    mats: sequence of (K, G, sigma_y, H[, n]) or Phase objects.
    """

    def __init__(self, N, phase, mats, precision="mixed", max_newton=50, max_cg=2000,
                 cg_inner_floor=1e-5, fixed_cg=0, fixed_newton=0, nrhs_tangent=6,
                 device=None, stream=None, cg_graph=1, dt=1.0, solver="cg"):
        import torch

        lib = load()
        self.N = int(N)
        self.V = self.N ** 3
        ph_arr = np.asarray(phase, dtype=np.uint8)
        self.ncells = 1 if ph_arr.ndim == 3 else int(ph_arr.shape[0])
        opt = default_options()
        opt.precision = FFTG_MIXED if precision == "mixed" else FFTG_FP64
        opt.max_newton = max_newton
        opt.max_cg = max_cg
        opt.cg_inner_floor = cg_inner_floor
        opt.fixed_cg = fixed_cg
        opt.fixed_newton = fixed_newton
        opt.nrhs_tangent = nrhs_tangent
        opt.cg_graph = cg_graph
        opt.dt = dt
        opt.solver = {"cg": FFTG_SOLVER_CG, "richardson": FFTG_SOLVER_RICHARDSON}[solver]
        self.device = torch.device(device or "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        b = C.c_size_t(0)
        check(lib.fftg_workspace_size_batch(self.N, self.ncells, C.byref(opt), C.byref(b)),
              "fftg_workspace_size_batch")
        nbytes = b.value
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        opt.workspace = C.c_void_p((base + 255) & ~255)
        opt.workspace_bytes = nbytes
        self.precision = precision
        ph = np.ascontiguousarray(np.asarray(phase, dtype=np.uint8).reshape(-1))
        m = phase_array(mats)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.fftg_create_batch(C.byref(h), self.N, self.ncells,
                                        ph.ctypes.data_as(C.POINTER(C.c_uint8)),
                                        len(mats), m, C.byref(opt)), "fftg_create_batch")
        self.h = h
        self._lib = lib

    def close(self):
        if getattr(self, "h", None):
            self._lib.fftg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Algorithm 1 --------------------------------------------------------
    def step(self, dE, tol_newton, tol_cg):
        dE = np.ascontiguousarray(dE, dtype=np.float64).reshape(6)
        sig = np.zeros(6)
        nn, nc = C.c_int(0), C.c_int(0)
        check(self._lib.fftg_step(self.h, _dptr(dE), tol_newton, tol_cg, _dptr(sig),
                                  C.byref(nn), C.byref(nc)), "fftg_step")
        return sig, nn.value, nc.value

    def batch_step(self, dE, tol_newton, tol_cg):
        """One increment for every cell: dE [ncells, 6] -> (sigma [ncells, 6],
        newton [ncells], cg [ncells], status [ncells])."""
        B = self.ncells
        dE = np.ascontiguousarray(dE, dtype=np.float64).reshape(B, 6)
        sig = np.zeros((B, 6))
        nn = (C.c_int * B)()
        nc = (C.c_int * B)()
        st = (C.c_int * B)()
        rc = self._lib.fftg_batch_step(self.h, dE.ctypes.data_as(_D6), tol_newton, tol_cg,
                                       sig.ctypes.data_as(_D6), nn, nc, st)
        if rc not in (FFTG_OK, FFTG_ENOCONV_NEWTON, FFTG_ENAN):
            check(rc, "fftg_batch_step")
        return sig, np.array(nn[:]), np.array(nc[:]), np.array(st[:])

    def select(self, cell):
        check(self._lib.fftg_select_cell(self.h, int(cell)), "fftg_select_cell")

    def stats(self):
        s = fftg_stats()
        check(self._lib.fftg_last_stats(self.h, C.byref(s)), "fftg_last_stats")
        n = min(s.newton_iters, FFTG_MAX_NEWTON_LOG)
        return dict(status=s.status, newton_iters=s.newton_iters, cg_iters=s.cg_iters,
                    cg_per_newton=list(s.cg_per_newton[:n]),
                    newton_norm=list(s.newton_norm[:n]), residual=list(s.residual[:n]),
                    cg_relres=list(s.cg_relres[:n]), cg_status=list(s.cg_status[:n]))

    def tangent(self, tol_cg):
        out = np.zeros(36)
        nc = C.c_int(0)
        check(self._lib.fftg_tangent(self.h, tol_cg, _dptr(out), C.byref(nc)), "fftg_tangent")
        return out.reshape(6, 6), nc.value

    # -- state --------------------------------------------------------------
    def reset_state(self):
        check(self._lib.fftg_reset_state(self.h), "fftg_reset_state")

    def get_state(self):
        n = self._lib.fftg_state_bytes(self.h)
        buf = np.zeros(n // 8)
        check(self._lib.fftg_get_state(self.h, buf.ctypes.data_as(C.c_void_p), n), "fftg_get_state")
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.float64)
        check(self._lib.fftg_set_state(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes),
              "fftg_set_state")

    def field(self, which):
        nc = {FFTG_FIELD_EPBAR: 1, FFTG_FIELD_TANGENT: 7}.get(which, 6)
        out = np.zeros(nc * self.V)
        check(self._lib.fftg_get_field(self.h, which, _dptr(out)), "fftg_get_field")
        return out.reshape((self.N,) * 3 if nc == 1 else (nc,) + (self.N,) * 3)

    # -- operators on device tensors ---------------------------------------
    def project(self, tau, out=None, dd=False):
        """G tau for a device tensor with 6 * N^3 elements (float64 or
        float32); dd=True: float64 buffers, double-float FFTs."""
        import torch
        assert tau.is_cuda and tau.is_contiguous() and tau.numel() == 6 * self.V
        prec = FFTG_FP64 if tau.dtype == torch.float64 else FFTG_MIXED
        if dd:
            assert tau.dtype == torch.float64
            prec = FFTG_DD
        if out is None:
            out = torch.empty_like(tau)
        check(self._lib.fftg_op_project(self.h, prec, C.c_void_p(tau.data_ptr()),
                                        C.c_void_p(out.data_ptr())), "fftg_op_project")
        return out

    def constitutive(self, dE=None, eps=None, sigma=None):
        import torch
        d = None if dE is None else np.ascontiguousarray(dE, dtype=np.float64).reshape(6)
        if sigma is None:
            sigma = torch.empty(6 * self.V, dtype=torch.float64, device=self.device)
        check(self._lib.fftg_op_constitutive(
            self.h, None if d is None else _dptr(d),
            None if eps is None else C.c_void_p(eps.data_ptr()),
            C.c_void_p(sigma.data_ptr())), "fftg_op_constitutive")
        return sigma

    # -- profiling ------------------------------------------------------------
    def profile(self, on=True):
        check(self._lib.fftg_profile_enable(self.h, 1 if on else 0), "fftg_profile_enable")

    def profile_reset(self):
        check(self._lib.fftg_profile_reset(self.h), "fftg_profile_reset")

    def profile_read(self):
        """{kernel kind name: (total device ms, launches)} since the last reset."""
        out = {}
        for k in range(self._lib.fftg_profile_kinds()):
            ms, n = C.c_double(0.0), C.c_longlong(0)
            check(self._lib.fftg_profile_read(self.h, k, C.byref(ms), C.byref(n)), "fftg_profile_read")
            if n.value:
                out[self._lib.fftg_profile_name(k).decode()] = (ms.value, n.value)
        return out

    def launch_count(self):
        return self._lib.fftg_launch_count(self.h)

    def matvec(self, p, q=None):
        import torch
        prec = FFTG_FP64 if p.dtype == torch.float64 else FFTG_MIXED
        if q is None:
            q = torch.empty_like(p)
        pq = C.c_double(0.0)
        check(self._lib.fftg_op_matvec(self.h, prec, C.c_void_p(p.data_ptr()),
                                       C.c_void_p(q.data_ptr()), C.byref(pq)), "fftg_op_matvec")
        return q, pq.value


class Group:
    """Several batch handles (`Cell`s, one grid size each) that take their
    increments together as one CUDA graph launch (fftg_group_*): Newton and
    CG loops run on the device, the handles' branches concurrently. The
    cells must outlive the group."""

    def __init__(self, cells):
        lib = load()
        self.cells = list(cells)
        arr = (C.c_void_p * len(self.cells))(*[c.h.value for c in self.cells])
        h = C.c_void_p()
        check(lib.fftg_group_create(C.byref(h), arr, len(self.cells)), "fftg_group_create")
        self.h = h
        self._lib = lib
        self.sizes = [c.ncells for c in self.cells]

    def step(self, dE, tol_newton, tol_cg, run=None):
        """One increment for every cell: dE is a list with one [ncells, 6]
        array per handle. Returns per handle (sigma [ncells, 6], newton,
        cg, status)."""
        tot = sum(self.sizes)
        d = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1, 6) for x in dE]))
        assert d.shape == (tot, 6)
        sig = np.zeros((tot, 6))
        nn = (C.c_int * tot)()
        nc = (C.c_int * tot)()
        st = (C.c_int * tot)()
        rp = None
        if run is not None:
            r = np.concatenate([np.asarray(x, dtype=np.int32).reshape(-1) for x in run])
            rp = (C.c_int * tot)(*[int(v) for v in r])
        rc = self._lib.fftg_group_step(self.h, d.ctypes.data_as(_D6), rp, tol_newton, tol_cg,
                                       sig.ctypes.data_as(_D6), nn, nc, st)
        if rc not in (FFTG_OK, FFTG_ENOCONV_NEWTON, FFTG_ENAN):
            check(rc, "fftg_group_step")
        out, o = [], 0
        for n in self.sizes:
            out.append((sig[o:o + n], np.array(nn[o:o + n]), np.array(nc[o:o + n]), np.array(st[o:o + n])))
            o += n
        return out

    def launch_count(self):
        return self._lib.fftg_group_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            self._lib.fftg_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server for one grid size (fftg_server_* calls).

    slots: cells held on the device (size them from the HBM budget with
    `workspace_size_batch`); sessions beyond that are evicted to host memory.
    """

    def __init__(self, N, slots, mats, precision="mixed", tol_newton=1e-5, tol_cg=1e-8,
                 max_newton=50, max_cg=2000, cg_inner_floor=1e-5, cg_graph=1, dt=1.0):
        lib = load()
        self.N = int(N)
        opt = default_options()
        opt.dt = dt
        opt.precision = FFTG_MIXED if precision == "mixed" else FFTG_FP64
        opt.max_newton = max_newton
        opt.max_cg = max_cg
        opt.cg_inner_floor = cg_inner_floor
        opt.nrhs_tangent = 0
        opt.cg_graph = cg_graph
        m = phase_array(mats)
        h = C.c_void_p()
        check(lib.fftg_server_start(C.byref(h), self.N, int(slots), len(mats), m, C.byref(opt),
                                    tol_newton, tol_cg), "fftg_server_start")
        self.h = h
        self._lib = lib
        self._buf = (fftg_result * 256)()

    @staticmethod
    def clock():
        return load().fftg_server_clock()

    def submit(self, request_id, session_id, dE, phase=None):
        dE = np.ascontiguousarray(dE, dtype=np.float64).reshape(6)
        ph = None
        if phase is not None:
            ph = np.ascontiguousarray(np.asarray(phase, dtype=np.uint8).reshape(-1))
        check(self._lib.fftg_server_submit(
            self.h, int(request_id), int(session_id),
            None if ph is None else ph.ctypes.data_as(C.POINTER(C.c_uint8)), _dptr(dE)),
            "fftg_server_submit")

    def poll(self, wait_s=0.0):
        n = C.c_int(0)
        check(self._lib.fftg_server_poll(self.h, self._buf, 256, C.byref(n), wait_s), "fftg_server_poll")
        out = []
        for i in range(n.value):
            r = self._buf[i]
            out.append(dict(request_id=r.request_id, session_id=r.session_id, status=r.status,
                            newton_iters=r.newton_iters, cg_iters=r.cg_iters, sigma=list(r.sigma),
                            t_submit=r.t_submit, t_start=r.t_start, t_done=r.t_done))
        return out

    def cancel_pending(self):
        """Drop the requests not yet admitted; returns how many."""
        n = C.c_longlong(0)
        check(self._lib.fftg_server_cancel_pending(self.h, C.byref(n)), "fftg_server_cancel_pending")
        return n.value

    def info(self):
        c, e, r = C.c_longlong(0), C.c_longlong(0), C.c_longlong(0)
        mc = C.c_int(0)
        mb = np.zeros(1)
        check(self._lib.fftg_server_info(self.h, C.byref(c), C.byref(e), C.byref(r), C.byref(mc),
                                         mb.ctypes.data_as(_D6)), "fftg_server_info")
        return dict(completed=c.value, evictions=e.value, restores=r.value,
                    max_concurrent=mc.value, mean_batch=float(mb[0]))

    def stop(self):
        if getattr(self, "h", None):
            rc = self._lib.fftg_server_stop(self.h)
            self.h = None
            check(rc, "fftg_server_stop")

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


class FsCell:
    """A finite-strain handle (include/fftg_fs.h): one periodic cell of
    St. Venant-Kirchhoff phases loaded by a macroscopic deformation gradient.

    phase: uint8 [N, N, N]; mats: (lambda, mu) pairs or objects with
    as_tuple(). Tensors are 3x3 (row major in the C calls)."""

    def __init__(self, N, phase, mats, precision="mixed", max_newton=50, max_cg=2000,
                 cg_inner_floor=1e-5, fixed_cg=0, fixed_newton=0, device=None, stream=None,
                 cg_graph=1):
        import torch

        lib = load()
        self.N = int(N)
        self.V = self.N ** 3
        opt = default_options()
        opt.precision = FFTG_MIXED if precision == "mixed" else FFTG_FP64
        opt.max_newton = max_newton
        opt.max_cg = max_cg
        opt.cg_inner_floor = cg_inner_floor
        opt.fixed_cg = fixed_cg
        opt.fixed_newton = fixed_newton
        opt.cg_graph = cg_graph
        self.device = torch.device(device or "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        self.precision = precision
        ph = np.ascontiguousarray(np.asarray(phase, dtype=np.uint8).reshape(-1))
        m = svk_array(mats)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.fftg_fs_create(C.byref(h), self.N, ph.ctypes.data_as(C.POINTER(C.c_uint8)),
                                     len(mats), m, C.byref(opt)), "fftg_fs_create")
        self.h = h
        self._lib = lib

    def close(self):
        if getattr(self, "h", None):
            self._lib.fftg_fs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dF, tol_newton, tol_cg):
        """One increment: Fbar += dF (3x3); returns (mean P 3x3, Newton
        iterations, CG iterations)."""
        dF = np.ascontiguousarray(dF, dtype=np.float64).reshape(9)
        P = np.zeros(9)
        nn, nc = C.c_int(0), C.c_int(0)
        check(self._lib.fftg_fs_step(self.h, _dptr(dF), tol_newton, tol_cg, _dptr(P),
                                     C.byref(nn), C.byref(nc)), "fftg_fs_step")
        return P.reshape(3, 3), nn.value, nc.value

    def stats(self):
        s = fftg_stats()
        check(self._lib.fftg_fs_last_stats(self.h, C.byref(s)), "fftg_fs_last_stats")
        n = min(s.newton_iters, FFTG_MAX_NEWTON_LOG)
        return dict(status=s.status, newton_iters=s.newton_iters, cg_iters=s.cg_iters,
                    cg_per_newton=list(s.cg_per_newton[:n]),
                    newton_norm=list(s.newton_norm[:n]), residual=list(s.residual[:n]),
                    cg_relres=list(s.cg_relres[:n]), cg_status=list(s.cg_status[:n]))

    def get_state(self):
        """Committed state: Fbar (9) then F* (9 N^3), FP64."""
        n = self._lib.fftg_fs_state_bytes(self.h)
        buf = np.zeros(n // 8)
        check(self._lib.fftg_fs_get_state(self.h, buf.ctypes.data_as(C.c_void_p), n), "fftg_fs_get_state")
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.float64)
        check(self._lib.fftg_fs_set_state(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes),
              "fftg_fs_set_state")

    def tangent(self, tol_cg):
        """9x9 macroscopic tangent dPbar/dFbar at the committed state
        (row 3i+j, column 3k+l) and the CG iterations of its nine solves."""
        out = np.zeros(81)
        nc = C.c_int(0)
        check(self._lib.fftg_fs_tangent(self.h, tol_cg, _dptr(out), C.byref(nc)), "fftg_fs_tangent")
        return out.reshape(9, 9), nc.value

    def field(self, which):
        out = np.zeros(9 * self.V)
        check(self._lib.fftg_fs_get_field(self.h, which, _dptr(out)), "fftg_fs_get_field")
        return out.reshape((3, 3) + (self.N,) * 3)

    def project(self, A, out=None, dd=False):
        """G A for a device tensor A with 9 * N^3 elements (float64 or
        float32); dd=True: float64 buffers, double-float FFTs."""
        import torch
        assert A.is_cuda and A.is_contiguous() and A.numel() == 9 * self.V
        prec = FFTG_FP64 if A.dtype == torch.float64 else FFTG_MIXED
        if dd:
            assert A.dtype == torch.float64
            prec = FFTG_DD
        if out is None:
            out = torch.empty_like(A)
        check(self._lib.fftg_fs_op_project(self.h, prec, C.c_void_p(A.data_ptr()),
                                           C.c_void_p(out.data_ptr())), "fftg_fs_op_project")
        return out

    def matvec(self, p, q=None):
        """q = G (K : p) at the committed state; returns (q, <p, q>)."""
        import torch
        assert p.is_cuda and p.is_contiguous() and p.numel() == 9 * self.V
        prec = FFTG_FP64 if p.dtype == torch.float64 else FFTG_MIXED
        if q is None:
            q = torch.empty_like(p)
        pq = C.c_double(0.0)
        check(self._lib.fftg_fs_op_matvec(self.h, prec, C.c_void_p(p.data_ptr()),
                                          C.c_void_p(q.data_ptr()), C.byref(pq)), "fftg_fs_op_matvec")
        return q, pq.value

    def profile(self, on=True):
        check(self._lib.fftg_fs_profile_enable(self.h, int(bool(on))), "fftg_fs_profile_enable")

    def profile_read(self):
        """{kernel kind name: (total device ms, launches)} since profiling was enabled."""
        out = {}
        for k in range(self._lib.fftg_fs_profile_kinds()):
            ms, n = C.c_double(0.0), C.c_longlong(0)
            check(self._lib.fftg_fs_profile_read(self.h, k, C.byref(ms), C.byref(n)),
                  "fftg_fs_profile_read")
            if n.value:
                out[self._lib.fftg_fs_profile_name(k).decode()] = (ms.value, n.value)
        return out

    def launches(self):
        return int(self._lib.fftg_fs_launch_count(self.h))


def fma_rate(precision="fp64", iters=1 << 16, stream=None):
    """Measured FMA throughput of the current device in TFLOP/s (FP64 or
    FP32), by the library's probe kernel (fftg_probe_fma_rate)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double(0.0)
    check(load().fftg_probe_fma_rate(FFTG_FP64 if precision == "fp64" else FFTG_MIXED, int(iters),
                                     C.c_void_p(st.cuda_stream), C.byref(out)), "fftg_probe_fma_rate")
    return out.value


SCHED_KINDS = ("p1", "p2", "p3", "p4", "p5")
SCHED_VARIANTS = 4
FFTG_TUNE_CACHE = 1
FFTG_TUNE_FORCE = 2


def schedule_set(N, kind, variant):
    """Select schedule `variant` of pass `kind` (0-4 or "p1".."p5") at grid N."""
    k = SCHED_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    check(load().fftg_schedule_set(int(N), k, int(variant)), "fftg_schedule_set")


def schedule_get(N):
    """{kind: variant} in use at grid N."""
    return {k: load().fftg_schedule_get(int(N), i) for i, k in enumerate(SCHED_KINDS)}


def schedule_describe(N, kind, variant):
    k = SCHED_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    sh = (C.c_int * 5)()
    check(load().fftg_schedule_describe(int(N), k, int(variant), sh), "fftg_schedule_describe")
    return dict(split=(sh[0], sh[1]), rows=sh[2], cols=sh[3], blocks=sh[4])


def autotune(N, cache=True, force=False, stream=None):
    """Time every schedule of the FP32 CG passes at grid N and select the
    fastest. Returns ({kind: chosen variant}, {kind: [ms per variant]})."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    ms = np.zeros(len(SCHED_KINDS) * SCHED_VARIANTS)
    ch = (C.c_int * len(SCHED_KINDS))()
    flags = (FFTG_TUNE_CACHE if cache else 0) | (FFTG_TUNE_FORCE if force else 0)
    check(load().fftg_autotune(int(N), flags, C.c_void_p(st.cuda_stream), _dptr(ms), ch), "fftg_autotune")
    return ({k: ch[i] for i, k in enumerate(SCHED_KINDS)},
            {k: [float(v) for v in ms[i * SCHED_VARIANTS:(i + 1) * SCHED_VARIANTS]]
             for i, k in enumerate(SCHED_KINDS)})
