"""Thin ctypes binding of libmg.so (include/mg.h): argument marshalling only.

Every arithmetic step of the solver runs in the library's CUDA kernels; this
module converts numpy arrays (host, MG_HOST) or CUDA torch tensors (device,
MG_DEVICE) into pointers, passes torch's current CUDA stream, and lets torch
allocate the device workspace.  There is no CPU fallback: if the library is
missing the import fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

MG_OK, MG_EINVAL, MG_ECUDA, MG_ENOCONV, MG_EREJECT, MG_ENONFINITE, MG_ETIMEOUT, MG_ENOMEM = 0, -1, -2, -3, -4, -5, -6, -7
MG_HOST, MG_DEVICE = 0, 1
MG_FP64, MG_MIXED = 0, 1
_NAMES = {0: "MG_OK", -1: "MG_EINVAL", -2: "MG_ECUDA", -3: "MG_ENOCONV", -4: "MG_EREJECT",
          -5: "MG_ENONFINITE", -6: "MG_ETIMEOUT", -7: "MG_ENOMEM"}

_dp = ctypes.POINTER(ctypes.c_double)


class mg_grid(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("R", ctypes.c_double), ("z", _dp)]


class mg_params(ctypes.Structure):
    _fields_ = [("V_cathode", ctypes.c_double), ("V_anode", ctypes.c_double),
                ("mu_e", ctypes.c_double), ("D_e", ctypes.c_double),
                ("mu_p", ctypes.c_double), ("D_p", ctypes.c_double),
                ("table", _dp), ("table_rows", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("pressure_factor", ctypes.c_double),
                ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32), ("coarsest", ctypes.c_int32),
                ("max_vcycles", ctypes.c_int32), ("max_newton", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("eta", ctypes.c_double), ("newton_tol", ctypes.c_double), ("corr_limit_frac", ctypes.c_double),
                ("dt1", ctypes.c_double), ("dt_growth", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("n0", ctypes.c_double), ("use_graphs", ctypes.c_int32), ("fused_sweep", ctypes.c_int32),
                ("guess_dt_max", ctypes.c_double), ("guess_level", ctypes.c_int32),
                ("guess_dt_start", ctypes.c_double),
                ("coarse_kernel_n", ctypes.c_int32), ("coarse_kernel_ctas", ctypes.c_int32),
                ("coarse_kernel_threads", ctypes.c_int32), ("eta_adapt", ctypes.c_int32),
                ("nu_coarse_n", ctypes.c_int32), ("nu_coarse1", ctypes.c_int32), ("nu_coarse2", ctypes.c_int32),
                ("nu_tiny_n", ctypes.c_int32), ("nu_tiny1", ctypes.c_int32), ("nu_tiny2", ctypes.c_int32),
                ("chain_from", ctypes.c_int32), ("pdl", ctypes.c_int32), ("wall_dirichlet", ctypes.c_int32),
                ("newton_tol_rel", ctypes.c_double), ("full_jacobian", ctypes.c_int32),
                ("max_corrections", ctypes.c_int32), ("line_smoother", ctypes.c_int32)]


class mg_stats(ctypes.Structure):
    _fields_ = [("steps_accepted", ctypes.c_int32), ("steps_rejected", ctypes.c_int32),
                ("newton_iterations", ctypes.c_int32), ("vcycles", ctypes.c_int32),
                ("last_newton", ctypes.c_int32), ("rho", ctypes.c_double * 3),
                ("steady_rho", ctypes.c_double), ("dt_last", ctypes.c_double), ("sim_time", ctypes.c_double),
                ("coarse_steps", ctypes.c_int32), ("coarse_newton", ctypes.c_int32),
                ("coarse_vcycles", ctypes.c_int32)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "rho" else getattr(self, k)) for k, _ in self._fields_}


_lib = None

# exported symbols and their signatures: (restype, argtypes)
_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "mg_params_default": (None, [ctypes.POINTER(mg_params)]),
    "mg_workspace_bytes": (_sz, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_params)]),
    "mg_create": (_i, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_params), _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "mg_destroy": (None, [_vp]),
    "mg_last_error": (ctypes.c_char_p, [_vp]),
    "mg_set_state": (_i, [_vp, _vp, _vp, _vp, _i]),
    "mg_get_state": (_i, [_vp, _vp, _vp, _vp, _i]),
    "mg_set_old_state": (_i, [_vp, _vp, _vp, _vp, _i]),
    "mg_set_sources": (_i, [_vp, _vp, _vp, _i]),
    "mg_residual": (_i, [_vp, _d, _vp, _vp, _vp, _vp, _i]),
    "mg_jacobian_apply": (_i, [_vp, _d, _vp, _vp, _vp, _vp, _vp, _vp, _i]),
    "mg_linear_solve": (_i, [_vp, _d, _vp, _vp, _vp, _vp, _vp, _vp, _d, _i, _vp, _vp, _i]),
    "mg_step": (_i, [_vp, _d, _d, ctypes.POINTER(mg_stats)]),
    "mg_march": (_i, [_vp, _d, _d, ctypes.POINTER(mg_stats)]),
    "mg_solve_steady": (_i, [_vp, _d, ctypes.POINTER(mg_stats)]),
    "mg_get_stats": (_i, [_vp, ctypes.POINTER(mg_stats)]),
    "mg_reset_stats": (None, [_vp]),
    "mg_kernel_launches": (ctypes.c_uint64, []),
    "mg_set_smoother": (_i, [_vp, _i, _i, _i, _i, _i, _i]),
    "mg_set_level_sweeps": (_i, [_vp, _i, _i, _i]),
    "mg_profile_begin": (_i, [_vp, _i, _i]),
    "mg_profile_end": (_i, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "mg_probe_fp64_gflops": (ctypes.c_double, [_vp]),
    "mg_time_smoother": (_i, [_vp, _i, _i, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "mg_solve_steady_batch": (_i, [ctypes.POINTER(_vp), _i, _d, _i, _vp, _vp]),
    "mg_autotune": (_i, [_vp, _vp]),
    "mg_autotune_batch": (_i, [ctypes.POINTER(_vp), _i, _d, ctypes.POINTER(_i)]),
    "mg_solve_steady_guess": (_i, [_vp, _vp, _vp, _vp, _i, _d, ctypes.POINTER(mg_stats), ctypes.POINTER(_i)]),
    "mg_num_levels": (_i, [_vp]),
    "mg_residual_noalloc": (_i, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_params), _vp, _vp, _vp, _vp, _vp, _vp,
                                 _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp]),
}
MG_PROF_SMOOTH, MG_PROF_LINRES, MG_PROF_COEF, MG_PROF_RESIDUAL, MG_PROF_RESTRICT, MG_PROF_PROLONG = 1, 2, 3, 4, 5, 6
MG_PROF_COARSE, MG_PROF_COARSE_FACTOR = 7, 8


def lib_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_0811_4446_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class MGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def default_params(**kw) -> mg_params:
    p = mg_params()
    load().mg_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "table":
            continue
        setattr(p, k, v)
    return p


def _torch():
    import torch
    return torch


def _ptr(a):
    """(pointer, where) of a numpy array (host) or a torch tensor (device or host)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float64")
        return a.ctypes.data, MG_HOST
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr(), (MG_DEVICE if a.is_cuda else MG_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def _where(*arrays):
    ws = {w for _, w in (_ptr(a) for a in arrays if a is not None)}
    if len(ws) != 1:
        raise TypeError("all arrays of one call must live in the same memory space")
    return ws.pop()


class Solver:
    """One discharge: an mg_state on the current CUDA device, workspace owned by a torch tensor."""

    def __init__(self, nr: int, nz: int, R: float, z, params: Optional[mg_params] = None, table=None,
                 stream=None, workspace: str = "torch"):
        self.lib = load()
        torch = _torch()
        self.nr, self.nz = int(nr), int(nz)
        self._z = np.ascontiguousarray(z, dtype=np.float64)
        if self._z.shape != (self.nz + 1,):
            raise ValueError("z must have nz + 1 entries")
        self.grid = mg_grid(self.nr, self.nz, float(R), self._z.ctypes.data_as(_dp))
        self.params = params if params is not None else default_params()
        self._table = None
        if table is not None:
            self._table = np.ascontiguousarray(table, dtype=np.float64)
            self.params.table = self._table.ctypes.data_as(_dp)
            self.params.table_rows = self._table.shape[0]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = self.lib.mg_workspace_bytes(ctypes.byref(self.grid), ctypes.byref(self.params))
        if nbytes == 0:
            raise MGError(MG_EINVAL, "invalid grid or parameters")
        self._ws = None
        ws_ptr = None
        if workspace == "torch":
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            ws_ptr = (base + 255) & ~255
        h = ctypes.c_void_p()
        rc = self.lib.mg_create(ctypes.byref(self.grid), ctypes.byref(self.params),
                                ctypes.c_void_p(self.stream.cuda_stream), ws_ptr, nbytes, ctypes.byref(h))
        if rc != MG_OK:
            raise MGError(rc, "mg_create failed")
        self.h = h
        self.shape = (self.nz + 1, self.nr + 1)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != MG_OK and rc not in allow:
            raise MGError(rc, self.lib.mg_last_error(self.h).decode())
        return rc

    # ---- state ------------------------------------------------------------------------
    def set_state(self, ne, np_, V):
        w = _where(ne, np_, V)
        self._check(self.lib.mg_set_state(self.h, _ptr(ne)[0], _ptr(np_)[0], _ptr(V)[0], w))

    def set_old_state(self, ne, np_, V):
        w = _where(ne, np_, V)
        self._check(self.lib.mg_set_old_state(self.h, _ptr(ne)[0], _ptr(np_)[0], _ptr(V)[0], w))

    def set_sources(self, S_e, S_p):
        w = _where(S_e, S_p)
        self._check(self.lib.mg_set_sources(self.h, _ptr(S_e)[0], _ptr(S_p)[0], w))

    def get_state(self, out=None):
        if out is None:
            out = [np.empty(self.shape) for _ in range(3)]
        w = _where(*out)
        self._check(self.lib.mg_get_state(self.h, *(_ptr(a)[0] for a in out), w))
        return out

    # ---- operators --------------------------------------------------------------------
    def residual(self, dt: float, with_F: bool = True):
        F = [np.empty(self.shape) for _ in range(3)] if with_F else [None, None, None]
        rho = (ctypes.c_double * 3)()
        ptrs = [(_ptr(a)[0] if a is not None else None) for a in F]
        self._check(self.lib.mg_residual(self.h, float(dt), *ptrs, rho, MG_HOST))
        return (F if with_F else None), np.array(rho[:])

    def jacobian_apply(self, dt: float, v: Sequence[np.ndarray]):
        out = [np.empty(self.shape) for _ in range(3)]
        v = [np.ascontiguousarray(a, dtype=np.float64) for a in v]
        self._check(self.lib.mg_jacobian_apply(self.h, float(dt), *(a.ctypes.data for a in v),
                                               *(a.ctypes.data for a in out), MG_HOST))
        return out

    def linear_solve(self, dt: float, f: Sequence[np.ndarray], eta: float, max_cycles: int):
        f = [np.ascontiguousarray(a, dtype=np.float64) for a in f]
        x = [np.empty(self.shape) for _ in range(3)]
        hist = np.zeros(max_cycles + 1)
        cyc = ctypes.c_int(0)
        rc = self.lib.mg_linear_solve(self.h, float(dt), *(a.ctypes.data for a in f), *(a.ctypes.data for a in x),
                                      float(eta), int(max_cycles), hist.ctypes.data, ctypes.byref(cyc), MG_HOST)
        self._check(rc, allow=(MG_ENOCONV,))
        return x, hist[:cyc.value + 1], rc

    # ---- drivers ------------------------------------------------------------------------
    def step(self, dt: float, tol: float):
        st = mg_stats()
        rc = self.lib.mg_step(self.h, float(dt), float(tol), ctypes.byref(st))
        self._check(rc, allow=(MG_ENOCONV, MG_ENONFINITE))
        return rc, st.as_dict()

    def march(self, dt_start: float, tol: float):
        st = mg_stats()
        rc = self.lib.mg_march(self.h, float(dt_start), float(tol), ctypes.byref(st))
        self._check(rc, allow=(MG_EREJECT,))
        return rc, st.as_dict()

    def solve_steady(self, tol: float):
        st = mg_stats()
        rc = self.lib.mg_solve_steady(self.h, float(tol), ctypes.byref(st))
        self._check(rc, allow=(MG_EREJECT,))
        return rc, st.as_dict()

    def solve_steady_guess(self, ne, np_, V, tol: float):
        """Steady solve from a full-grid guess; returns (rc, stats, used_fallback)."""
        st = mg_stats()
        fb = ctypes.c_int(0)
        w = _where(ne, np_, V)
        rc = self.lib.mg_solve_steady_guess(self.h, _ptr(ne)[0], _ptr(np_)[0], _ptr(V)[0], w, float(tol),
                                            ctypes.byref(st), ctypes.byref(fb))
        self._check(rc, allow=(MG_EREJECT,))
        return rc, st.as_dict(), bool(fb.value)

    def stats(self):
        st = mg_stats()
        self._check(self.lib.mg_get_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def reset_stats(self):
        self.lib.mg_reset_stats(self.h)

    def set_smoother(self, level: int, precision: int, bx: int, by: int, fused: int, tile: int):
        """Smoother launch of one level by hand (see mg_set_smoother in include/mg.h)."""
        self._check(self.lib.mg_set_smoother(self.h, level, precision, bx, by, fused, tile))

    def set_level_sweeps(self, level: int, nu1: int, nu2: int):
        """Sweeps of one level by hand (see mg_set_level_sweeps in include/mg.h)."""
        self._check(self.lib.mg_set_level_sweeps(self.h, level, nu1, nu2))

    def autotune(self):
        n = self.lib.mg_num_levels(self.h)
        out = np.zeros(6 * n, dtype=np.int32)
        self._check(self.lib.mg_autotune(self.h, out.ctypes.data))
        return out.reshape(n, 6)

    def time_smoother(self, level: int, precision: int = 0, sweeps: int = 200):
        """(device us per smoother launch, launches per sweep) with the level's sweeps replayed
        from a captured graph (see mg_time_smoother in include/mg.h)."""
        us = ctypes.c_double(0.0)
        lps = ctypes.c_int(0)
        self._check(self.lib.mg_time_smoother(self.h, int(level), int(precision), int(sweeps), ctypes.byref(us),
                                              ctypes.byref(lps)))
        return us.value, lps.value

    def profile_begin(self, kernel: int, level: int = 0):
        self._check(self.lib.mg_profile_begin(self.h, int(kernel), int(level)))

    def profile_end(self):
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        self._check(self.lib.mg_profile_end(self.h, ctypes.byref(n), ctypes.byref(ms)))
        return int(n.value), float(ms.value)


def solve_steady_batch(solvers, tol: float, workers: int = 0):
    """Steady solves of independent Solver objects; returns (rc, ms[n], rc[n]).

    workers = 0: the batched persistent launch (every discharge's whole steady solve in one
    launch); workers > 0: that many host threads solving the discharges one by one (the
    comparison form).  See mg_solve_steady_batch in include/mg.h."""
    lib = load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.h for s in solvers])
    ms = np.zeros(n)
    rcs = np.zeros(n, dtype=np.int32)
    rc = lib.mg_solve_steady_batch(hs, n, float(tol), int(workers), ms.ctypes.data, rcs.ctypes.data)
    return rc, ms, rcs


def autotune_batch(solvers, tol: float):
    """Work list of the persistent batched form tuned on these discharges (see
    mg_autotune_batch in include/mg.h); returns (work-item size, coarse-phase level) kept."""
    lib = load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.h for s in solvers])
    g = ctypes.c_int(0)
    rc = lib.mg_autotune_batch(hs, n, float(tol), ctypes.byref(g))
    if rc != MG_OK:
        raise MGError(rc, "mg_autotune_batch failed")
    return g.value % 100, g.value // 100


def residual_noalloc(nr: int, nz: int, R: float, z, params: mg_params, state, old_state, sources, dt: float,
                     F_out=None, table=None, stream=None):
    """rho[3] (and optionally the residual rows into F_out) through mg_residual_noalloc.

    state, old_state (or None when dt <= 0), sources and F_out are CUDA float64 tensors of
    shape (nz + 1, nr + 1); nothing is allocated on the device by the call.
    """
    torch = _torch()
    lib = load()
    zh = np.ascontiguousarray(z, dtype=np.float64)
    grid = mg_grid(int(nr), int(nz), float(R), zh.ctypes.data_as(_dp))
    keep = None
    if table is not None:
        keep = np.ascontiguousarray(table, dtype=np.float64)
        params.table = keep.ctypes.data_as(_dp)
        params.table_rows = keep.shape[0]
    ptr = lambda a: None if a is None else _ptr(a)[0]
    old = old_state if old_state is not None else (None, None, None)
    F = F_out if F_out is not None else (None, None, None)
    rho = (ctypes.c_double * 3)()
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.mg_residual_noalloc(ctypes.byref(grid), ctypes.byref(params), *(ptr(a) for a in state),
                                 *(ptr(a) for a in old), *(ptr(a) for a in sources), float(dt),
                                 *(ptr(a) for a in F), rho, ctypes.c_void_p(st.cuda_stream))
    del keep
    if rc != MG_OK:
        raise MGError(rc, "mg_residual_noalloc failed")
    return np.array(rho[:])


def kernel_launches() -> int:
    return int(load().mg_kernel_launches())


def probe_fp64_gflops() -> float:
    torch = _torch()
    return float(load().mg_probe_fp64_gflops(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))


def from_discharge(d, stream=None, **param_overrides) -> Solver:
    """Solver for a workloads.Discharge (sources and initial state loaded)."""
    kw = dict(V_cathode=d.V_cathode, V_anode=d.V_anode, mu_e=d.mu_e, D_e=d.D_e, mu_p=d.mu_p, D_p=d.D_p,
              pressure_factor=d.pressure_factor, wall_dirichlet=int(getattr(d, "wall_dirichlet", False)))
    kw.update(param_overrides)
    p = default_params(**kw)
    s = Solver(d.nr, d.nz, d.R, d.z, p, table=d.table, stream=stream)
    s.set_sources(np.ascontiguousarray(d.S_e), np.ascontiguousarray(d.S_p))
    s.set_state(np.ascontiguousarray(d.ne0), np.ascontiguousarray(d.np0), np.ascontiguousarray(d.V0))
    return s
