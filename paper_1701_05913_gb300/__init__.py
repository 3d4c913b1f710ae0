"""Python binding of the GB300 preconditioned Krylov library (librs.so).

Argument marshalling only: every step of the solve runs in the CUDA kernels
of librs.so, reached through the C ABI declared in include/rs.h.  PyTorch
supplies device memory (tensors) and the CUDA stream.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

Raw entry points keep their C names (``rs_init``, ``rs_mat_create_csr``,
``rs_solve_gmres`` ...) on the loaded library object returned by ``lib()``;
the classes below wrap the handles.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "librs.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_BAD_PATTERN, ERR_ZERO_PIVOT, ERR_BREAKDOWN = -1, -2, -3, -4
ERR_DEVICE_TIMEOUT, ERR_CUDA, ERR_OOM, ERR_SIZE_MISMATCH = -5, -6, -7, -8
MEM_HOST, MEM_DEVICE = 0, 1
PC_NONE, PC_ILU0, PC_BILU0, PC_CPR, PC_CPR_LEARNED, PC_RAS, PC_AMG = 0, 1, 2, 3, 4, 5, 6
FP64, MIXED = 0, 1

_PC_KIND = {"none": PC_NONE, "ilu0": PC_ILU0, "bilu0": PC_BILU0, "cpr": PC_CPR,
            "cpr_learned": PC_CPR_LEARNED, "ras": PC_RAS, "amg": PC_AMG}


def box_partition(grid, parts):
    """Subdomain of every cell of an nx x ny x nz grid (x fastest) cut into
    px x py x pz boxes of near-equal size: the row partition that gives
    restricted additive Schwarz compact subdomains."""
    (nx, ny, nz), (px, py, pz) = grid, parts
    bx = np.arange(nx) * px // nx
    by = np.arange(ny) * py // ny
    bz = np.arange(nz) * pz // nz
    return ((bz[:, None, None] * py + by[None, :, None]) * px + bx[None, None, :]).reshape(-1).astype(np.int32)

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_f32p = C.POINTER(C.c_float)
_vp = C.c_void_p


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("status", C.c_int32),
                ("bad_row", C.c_int32), ("true_rel_res", C.c_double),
                ("implicit_rel_res", C.c_double), ("solve_s", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PcOpts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("net", _vp), ("log_perm", _vp), ("cpr_form", C.c_int32),
                ("ras_nparts", C.c_int32), ("ras_overlap", C.c_int32), ("ilu_level", C.c_int32),
                ("ras_part", _vp), ("amg_theta", C.c_double), ("amg_max_levels", C.c_int32),
                ("amg_max_coarse", C.c_int32), ("amg_nu", C.c_int32), ("cpr_pstage", C.c_int32),
                ("ras_local", C.c_int32), ("ilut_p", C.c_int32), ("ilut_tol", C.c_double),
                ("amg_smoother", C.c_int32), ("sweep", C.c_int32), ("sweep_run_cap", C.c_int32)]


CPR_FORMS = ("pf", "fp", "fpf", "ffpf")   # rs_cpr_form: Algs. 6, 5, 7, 8


# (name, restype, argtypes) for every exported symbol of include/rs.h
SIGNATURES = [
    ("rs_init", C.c_int, [C.POINTER(_vp), C.c_int, _vp]),
    ("rs_finalize", C.c_int, [C.POINTER(_vp)]),
    ("rs_sync", C.c_int, [_vp]),
    ("rs_set_spin_limit", C.c_int, [_vp, C.c_int64]),
    ("rs_set_history", C.c_int, [_vp, C.POINTER(C.c_double), C.c_int32]),
    ("rs_check_device", C.c_int, [_vp]),
    ("rs_status_str", C.c_char_p, [C.c_int]),
    ("rs_launch_count", C.c_int64, [_vp]),
    ("rs_prof_enable", C.c_int, [_vp, C.c_int]),
    ("rs_prof_read", C.c_int, [_vp, _f64p, C.POINTER(C.c_int64), C.c_int32, C.c_int]),
    ("rs_vec_create", C.c_int, [_vp, C.c_int32, C.POINTER(_vp)]),
    ("rs_vec_wrap", C.c_int, [_vp, C.c_int32, _vp, C.POINTER(_vp)]),
    ("rs_vec_destroy", C.c_int, [C.POINTER(_vp)]),
    ("rs_vec_size", C.c_int32, [_vp]),
    ("rs_vec_data", _vp, [_vp]),
    ("rs_vec_set", C.c_int, [_vp, _vp, C.c_int]),
    ("rs_vec_get", C.c_int, [_vp, _vp, C.c_int]),
    ("rs_vec_set_value", C.c_int, [_vp, C.c_double]),
    ("rs_vec_axpby", C.c_int, [C.c_double, _vp, C.c_double, _vp]),
    ("rs_vec_axpbyz", C.c_int, [C.c_double, _vp, C.c_double, _vp, _vp]),
    ("rs_vec_dot", C.c_int, [_vp, _vp, _f64p]),
    ("rs_vec_norm2", C.c_int, [_vp, _f64p]),
    ("rs_vec_mdot_noalloc", C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    ("rs_mat_create_csr", C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, C.c_int, C.POINTER(_vp)]),
    ("rs_mat_create_bsr", C.c_int, [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_int,
                                    C.POINTER(_vp)]),
    ("rs_mat_destroy", C.c_int, [C.POINTER(_vp)]),
    ("rs_mat_size", C.c_int32, [_vp]),
    ("rs_mat_spmv", C.c_int, [_vp, _vp, _vp]),
    ("rs_mat_amxpby", C.c_int, [C.c_double, _vp, _vp, C.c_double, _vp]),
    ("rs_precond_setup", C.c_int, [_vp, _vp, C.c_int, C.POINTER(PcOpts), C.POINTER(_vp)]),
    ("rs_precond_apply", C.c_int, [_vp, _vp, _vp]),
    ("rs_precond_get_ilu", C.c_int, [_vp, _f64p, C.c_int32]),
    ("rs_precond_get_bilu", C.c_int, [_vp, _f64p, _f64p]),
    ("rs_precond_get_cpr", C.c_int, [_vp, _f64p, _f64p]),
    ("rs_precond_bad_row", C.c_int32, [_vp]),
    ("rs_precond_sweep_levels", C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("rs_precond_sweep_kind", C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32)]),
    ("rs_precond_sweep_runs", C.c_int, [_vp] + [C.POINTER(C.c_int32)] * 4),
    ("rs_sweep_schedule", C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int32, C.c_int32,
                                    C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("rs_precond_ras_info", C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    ("rs_precond_amg_levels", C.c_int, [_vp, C.POINTER(C.c_int32)]),
    ("rs_precond_amg_level_sizes", C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                             C.POINTER(C.c_int64)]),
    ("rs_precond_get_amg_level", C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _f64p,
                                           C.POINTER(C.c_int32), C.POINTER(C.c_int32), _f64p,
                                           C.POINTER(C.c_int32)]),
    ("rs_precond_get_ras", C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     _f64p]),
    ("rs_precond_destroy", C.c_int, [C.POINTER(_vp)]),
    ("rs_solve_gmres", C.c_int, [_vp, _vp, _vp, _vp, C.c_int32, C.c_double, C.c_int32,
                                 C.POINTER(SolveInfo)]),
    ("rs_solve_fgmres", C.c_int, [_vp, _vp, _vp, _vp, C.c_int32, C.c_double, C.c_int32,
                                  C.POINTER(SolveInfo)]),
    ("rs_solve_lgmres", C.c_int, [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                  C.POINTER(SolveInfo)]),
    ("rs_solve_bicgstab", C.c_int, [_vp, _vp, _vp, _vp, C.c_double, C.c_int32,
                                    C.POINTER(SolveInfo)]),
    ("rs_solve_cg", C.c_int, [_vp, _vp, _vp, _vp, C.c_double, C.c_int32, C.POINTER(SolveInfo)]),
    ("rs_net_num_params", C.c_int64, []),
    ("rs_net_create", C.c_int, [_vp, _f32p, C.c_int64, C.c_float, C.POINTER(_vp)]),
    ("rs_net_destroy", C.c_int, [C.POINTER(_vp)]),
    ("rs_net_get_params", C.c_int, [_vp, _f32p, C.c_int64]),
    ("rs_net_get_grads", C.c_int, [_vp, _f32p, C.c_int64]),
    ("rs_net_zero_grads", C.c_int, [_vp]),
    ("rs_net_forward", C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp]),
    ("rs_net_accumulate", C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_double,
                                    C.POINTER(C.c_double)]),
    ("rs_net_adam", C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float]),
    ("rs_net_save", C.c_int, [_vp, C.c_char_p]),
    ("rs_net_load", C.c_int, [_vp, C.c_char_p, C.POINTER(_vp)]),
]

_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    from . import _build
    return _build.build(force=force, verbose=verbose)


def _finalizing() -> bool:
    """True once the interpreter is shutting down: finalizers then leave the
    handles to process exit (the driver reclaims the memory), because ctypes,
    torch and the CUDA runtime may already be half torn down."""
    return sys.is_finalizing()


def lib():
    """Loads librs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librs.so not built: run __graft_entry__.build() "
                              "(or python -m paper_1701_05913_gb300._build)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class RsError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = lib().rs_status_str(status).decode()
        super().__init__("%s failed: %s (%d)" % (what, msg, status))


def _check(status, what):
    if status != OK:
        raise RsError(status, what)


def _torch():
    import torch
    return torch


def _dev_f64(t):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t, dtype=np.float64))
    t = t.to(device="cuda", dtype=torch.float64).contiguous()
    return t


def _dev_i32(t):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t, dtype=np.int32))
    return t.to(device="cuda", dtype=torch.int32).contiguous()


class Context:
    """rs_init on a CUDA device and a stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("the CUDA library needs a GPU; none is visible")
        torch.cuda.set_device(device)
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.h = _vp()
        _check(lib().rs_init(C.byref(self.h), device, _vp(stream.cuda_stream)), "rs_init")

    def sync(self):
        _check(lib().rs_sync(self.h), "rs_sync")

    def launches(self) -> int:
        return lib().rs_launch_count(self.h)

    PROF_KINDS = ("spmv", "l_sweep", "u_sweep", "cgs_dots", "cgs_update_dots", "cgs_update_norm",
                  "blas1", "precond_other", "factor", "solver_scalar", "net", "bl_sweep", "bu_sweep",
                  "cpr_resid")

    def prof_enable(self, on=True):
        _check(lib().rs_prof_enable(self.h, int(on)), "rs_prof_enable")

    def prof_read(self, reset=True):
        k = len(self.PROF_KINDS)
        ms = (C.c_double * k)()
        cnt = (C.c_int64 * k)()
        _check(lib().rs_prof_read(self.h, ms, cnt, k, int(reset)), "rs_prof_read")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(self.PROF_KINDS)}

    def set_history(self, length: int):
        """Record the residual history of the following solves (up to
        `length` iterations each); length = 0 stops.  Returns the numpy array
        the solves write into (rs_set_history)."""
        if length <= 0:
            self._hist = None
            _check(lib().rs_set_history(self.h, None, 0), "rs_set_history")
            return None
        self._hist = np.full(length, np.nan)
        _check(lib().rs_set_history(self.h, self._hist.ctypes.data_as(C.POINTER(C.c_double)), length),
               "rs_set_history")
        return self._hist

    def set_spin_limit(self, cycles: int):
        """Clock cycles a device-side wait may take before it gives up (0: default)."""
        _check(lib().rs_set_spin_limit(self.h, cycles), "rs_set_spin_limit")

    def check(self) -> int:
        """Read and clear the device error word: OK or ERR_DEVICE_TIMEOUT, ..."""
        return lib().rs_check_device(self.h)

    def close(self):
        if self.h:
            lib().rs_finalize(C.byref(self.h))

    def __del__(self):
        try:
            if not _finalizing():
                self.close()
        except Exception:
            pass


class Vec:
    """An FP64 device vector viewing a torch tensor (rs_vec_wrap)."""

    def __init__(self, ctx: Context, t):
        self.ctx = ctx
        self.t = _dev_f64(t)
        self.n = self.t.numel()
        self.h = _vp()
        _check(lib().rs_vec_wrap(ctx.h, self.n, _vp(self.t.data_ptr()), C.byref(self.h)), "rs_vec_wrap")

    @classmethod
    def zeros(cls, ctx, n):
        return cls(ctx, _torch().zeros(n, dtype=_torch().float64, device="cuda"))

    def numpy(self):
        self.ctx.sync()
        return self.t.cpu().numpy()

    def __del__(self):
        try:
            if self.h and not _finalizing():
                lib().rs_vec_destroy(C.byref(self.h))
        except Exception:
            pass


class Mat:
    """CSR or BSR matrix handle (the library keeps its own device copy)."""

    def __init__(self, ctx: Context, ptr, col, val, bs: int = 1):
        self.ctx = ctx
        self.bs = int(bs)
        p, c, v = _dev_i32(ptr), _dev_i32(col), _dev_f64(val)
        self.nrows = p.numel() - 1
        self.n = self.nrows * self.bs
        self.h = _vp()
        if self.bs == 1:
            st = lib().rs_mat_create_csr(ctx.h, self.nrows, _vp(p.data_ptr()), _vp(c.data_ptr()),
                                         _vp(v.data_ptr()), MEM_DEVICE, C.byref(self.h))
        else:
            st = lib().rs_mat_create_bsr(ctx.h, self.nrows, self.bs, _vp(p.data_ptr()),
                                         _vp(c.data_ptr()), _vp(v.data_ptr()), MEM_DEVICE,
                                         C.byref(self.h))
        _check(st, "rs_mat_create")
        self.nnz = c.numel()

    @classmethod
    def csr(cls, ctx, m: dict):
        return cls(ctx, m["rowptr"], m["col"], m["val"], 1)

    @classmethod
    def bsr(cls, ctx, m: dict):
        return cls(ctx, m["browptr"], m["bcol"], m["bval"], m["bs"])

    def spmv(self, x: Vec, y: Vec):
        _check(lib().rs_mat_spmv(self.h, x.h, y.h), "rs_mat_spmv")

    def amxpby(self, a, x: Vec, b, y: Vec):
        _check(lib().rs_mat_amxpby(a, self.h, x.h, b, y.h), "rs_mat_amxpby")

    def __del__(self):
        try:
            if self.h and not _finalizing():
                lib().rs_mat_destroy(C.byref(self.h))
        except Exception:
            pass


class Precond:
    """rs_precond_setup / apply / destroy."""

    def __init__(self, ctx: Context, A: Mat, kind: str = "ilu0", prec: str = "fp64",
                 net=None, log_perm=None, grid=None, form: str = "pf", nparts: int = 1, part=None,
                 overlap: int = 0, level: int = 0, amg=None, pstage: str = "ilu0", ilut=None,
                 sweep: str = "auto", run_cap: int = 0):
        self.ctx, self.A, self.kind = ctx, A, kind
        opts = PcOpts()
        opts.prec = MIXED if prec == "mixed" else FP64
        opts.cpr_form = CPR_FORMS.index(form)
        self._keep = []
        if net is not None:
            opts.net = net.h.value
            lp = _dev_f64(log_perm)
            self._keep += [net, lp]
            opts.log_perm = lp.data_ptr()
            opts.nx, opts.ny, opts.nz = grid
        # restricted additive Schwarz: subdomains, overlap layers, ILU(k) level
        opts.ras_nparts, opts.ras_overlap, opts.ilu_level = nparts, overlap, level
        if ilut is not None:           # (p, tol): ILUT local solvers instead of ILU(level)
            opts.ras_local, opts.ilut_p, opts.ilut_tol = 1, ilut[0], ilut[1]
        # algebraic multigrid (kind "amg", or the CPR pressure stage with pstage="amg")
        a = amg or {}
        opts.amg_theta = a.get("theta", 0.0)
        opts.amg_max_levels = a.get("max_levels", 0)
        opts.amg_max_coarse = a.get("max_coarse", 0)
        opts.amg_nu = a.get("nu", 0)
        opts.amg_smoother = a.get("smoother", 0)
        opts.cpr_pstage = {"ilu0": 0, "amg": 1}[pstage]
        # ILU sweeps: "auto" (the library's choice), "segments" or "wavefront"
        # (structured 7-point grids; other patterns keep the segments)
        opts.sweep = {"auto": 0, "segments": 1, "wavefront": 2}[sweep]
        opts.sweep_run_cap = run_cap
        if part is not None:
            part = np.ascontiguousarray(part, dtype=np.int32)
            self._keep.append(part)
            opts.ras_part = part.ctypes.data
        self.h = _vp()
        self.status = lib().rs_precond_setup(ctx.h, A.h, _PC_KIND[kind], C.byref(opts), C.byref(self.h))
        self.bad_row = lib().rs_precond_bad_row(self.h) if self.h else -1
        if self.status != ERR_ZERO_PIVOT:
            _check(self.status, "rs_precond_setup")

    def apply(self, r: Vec, z: Vec):
        _check(lib().rs_precond_apply(self.h, r.h, z.h), "rs_precond_apply")

    def ilu_factors(self, nnz):
        out = np.empty(nnz)
        _check(lib().rs_precond_get_ilu(self.h, out.ctypes.data_as(_f64p), nnz), "rs_precond_get_ilu")
        return out

    def bilu_factors(self):
        bs = self.A.bs
        lu = np.empty(self.A.nnz * bs * bs)
        dinv = np.empty(self.A.nrows * bs * bs)
        _check(lib().rs_precond_get_bilu(self.h, lu.ctypes.data_as(_f64p), dinv.ctypes.data_as(_f64p)),
               "rs_precond_get_bilu")
        return lu, dinv

    def cpr_data(self):
        bs = self.A.bs
        w = np.empty(self.A.nrows * (bs - 1))
        app = np.empty(self.A.nnz)
        _check(lib().rs_precond_get_cpr(self.h, w.ctypes.data_as(_f64p), app.ctypes.data_as(_f64p)),
               "rs_precond_get_cpr")
        return w, app

    def amg_sizes(self):
        """AMG hierarchy sizes: [(rows of A_l, entries of A_l, entries of P_l)]."""
        L = lib()
        nl = C.c_int32()
        _check(L.rs_precond_amg_levels(self.h, C.byref(nl)), "rs_precond_amg_levels")
        out = []
        for l in range(nl.value):
            n, na, np_ = C.c_int32(), C.c_int64(), C.c_int64()
            _check(L.rs_precond_amg_level_sizes(self.h, l, C.byref(n), C.byref(na), C.byref(np_)),
                   "rs_precond_amg_level_sizes")
            out.append((n.value, na.value, np_.value))
        return out

    def amg_levels(self):
        """AMG hierarchy: per level dict(A=(ptr, col, val), P=(ptr, col, val)
        or None, cidx=coarse index per point or None)."""
        L = lib()
        nl = C.c_int32()
        _check(L.rs_precond_amg_levels(self.h, C.byref(nl)), "rs_precond_amg_levels")
        i32 = C.POINTER(C.c_int32)
        out = []
        for l in range(nl.value):
            n, na, np_ = C.c_int32(), C.c_int64(), C.c_int64()
            _check(L.rs_precond_amg_level_sizes(self.h, l, C.byref(n), C.byref(na), C.byref(np_)),
                   "rs_precond_amg_level_sizes")
            last = l + 1 == nl.value
            a = (np.empty(n.value + 1, np.int32), np.empty(na.value, np.int32), np.empty(na.value))
            p = None if last else (np.empty(n.value + 1, np.int32), np.empty(np_.value, np.int32),
                                   np.empty(np_.value))
            cidx = None if last else np.empty(n.value, np.int32)
            _check(L.rs_precond_get_amg_level(
                self.h, l, a[0].ctypes.data_as(i32), a[1].ctypes.data_as(i32), a[2].ctypes.data_as(_f64p),
                p[0].ctypes.data_as(i32) if p else None, p[1].ctypes.data_as(i32) if p else None,
                p[2].ctypes.data_as(_f64p) if p else None, cidx.ctypes.data_as(i32) if cidx is not None else None),
                "rs_precond_get_amg_level")
            out.append(dict(A=a, P=p, cidx=cidx))
        return out

    def ras_info(self):
        """RAS: (stacked rows, stored entries) of the extended subdomains."""
        ne, nz = C.c_int32(), C.c_int64()
        _check(lib().rs_precond_ras_info(self.h, C.byref(ne), C.byref(nz)), "rs_precond_ras_info")
        return ne.value, nz.value

    def ras_structure(self):
        """RAS: (gidx, ptr, col, lu) of the stacked extended subdomains."""
        ne, nz = C.c_int32(), C.c_int64()
        _check(lib().rs_precond_ras_info(self.h, C.byref(ne), C.byref(nz)), "rs_precond_ras_info")
        bs = self.A.bs
        gidx = np.empty(ne.value, np.int32)
        ptr = np.empty(ne.value + 1, np.int32)
        col = np.empty(nz.value, np.int32)
        lu = np.empty(nz.value * bs * bs)
        i32 = C.POINTER(C.c_int32)
        _check(lib().rs_precond_get_ras(self.h, gidx.ctypes.data_as(i32), ptr.ctypes.data_as(i32),
                                        col.ctypes.data_as(i32), lu.ctypes.data_as(_f64p)), "rs_precond_get_ras")
        return gidx, ptr, col, lu

    def sweep_levels(self):
        """(L levels, U levels) of the full-system factor's triangular sweeps."""
        a, b = C.c_int32(), C.c_int32()
        _check(lib().rs_precond_sweep_levels(self.h, C.byref(a), C.byref(b)), "rs_precond_sweep_levels")
        return a.value, b.value

    def sweep_kind(self):
        """("segments", None) or ("wavefront", (nx, ny, nz)) for the
        full-system factor's triangular sweeps."""
        v = [C.c_int32() for _ in range(4)]
        _check(lib().rs_precond_sweep_kind(self.h, *[C.byref(x) for x in v]), "rs_precond_sweep_kind")
        return ("wavefront", (v[1].value, v[2].value, v[3].value)) if v[0].value else ("segments", None)

    def sweep_runs(self):
        """(L runs, U runs, longest L run, longest U run) of the same sweeps."""
        v = [C.c_int32() for _ in range(4)]
        _check(lib().rs_precond_sweep_runs(self.h, *[C.byref(x) for x in v]), "rs_precond_sweep_runs")
        return tuple(x.value for x in v)

    def __del__(self):
        try:
            if self.h and not _finalizing():
                lib().rs_precond_destroy(C.byref(self.h))
        except Exception:
            pass


NET_LAYERS = [("e0a", 2), ("e0b", 16), ("e1a", 16), ("e1b", 16), ("e2a", 16), ("e2b", 16),
              ("e3a", 16), ("e3b", 16), ("d2a", 32), ("d2b", 16), ("d1a", 32), ("d1b", 16),
              ("d0a", 32), ("d0b", 16)]


def net_flatten(params: dict) -> np.ndarray:
    """Flat FP32 parameter vector in the layout rs_net_create expects, from a
    dict of arrays: name.W (3, 3, 3, 16, cin), name.b (16,), head.W (1, 16),
    head.b (1,)."""
    parts = []
    for name, cin in NET_LAYERS:
        parts += [np.asarray(params[name + ".W"]).reshape(-1), np.asarray(params[name + ".b"]).reshape(-1)]
    parts += [np.asarray(params["head.W"]).reshape(-1), np.asarray(params["head.b"]).reshape(-1)]
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)


def net_unflatten(flat) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    out, off = {}, 0
    for name, cin in NET_LAYERS:
        n = 27 * 16 * cin
        out[name + ".W"] = flat[off:off + n].reshape(3, 3, 3, 16, cin)
        off += n
        out[name + ".b"] = flat[off:off + 16].copy()
        off += 16
    out["head.W"] = flat[off:off + 16].reshape(1, 16)
    out["head.b"] = flat[off + 16:off + 17].copy()
    return out


def sweep_schedule(ptr, col, lower=True, run_cap=1 << 30, run_slots=1 << 40):
    """The host-side schedule of one triangular sweep of a CSR pattern
    (rs_sweep_schedule): segment first rows and levels, and the runs as
    rows of (first segment, segments, segment stride, row stride, entry
    stride), in ticket order.  Needs no GPU."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = ptr.size - 1
    nseg, nlev, nrun = C.c_int32(), C.c_int32(), C.c_int32()
    row0 = np.zeros(n + 1, np.int32)
    lev = np.zeros(max(n, 1), np.int32)
    runs = np.zeros(5 * max(n, 1), np.int32)
    i32 = C.POINTER(C.c_int32)
    _check(lib().rs_sweep_schedule(n, ptr.ctypes.data_as(i32), col.ctypes.data_as(i32), int(lower), run_cap,
                                   run_slots, C.byref(nseg), C.byref(nlev), C.byref(nrun), row0.ctypes.data_as(i32),
                                   lev.ctypes.data_as(i32), runs.ctypes.data_as(i32)), "rs_sweep_schedule")
    return dict(row0=row0[:nseg.value + 1].copy(), level=lev[:nseg.value].copy(), nlevels=nlev.value,
                runs=runs[:5 * nrun.value].reshape(-1, 5).copy())


class Net:
    """The learned pressure-stage network (rs_net_*)."""

    def __init__(self, ctx: Context, params: dict | None = None, out_scale: float = 1.0, path: str | None = None):
        self.ctx = ctx
        self.h = _vp()
        if path is not None:
            _check(lib().rs_net_load(ctx.h, path.encode(), C.byref(self.h)), "rs_net_load")
        else:
            flat = net_flatten(params)
            _check(lib().rs_net_create(ctx.h, flat.ctypes.data_as(_f32p), flat.size, out_scale, C.byref(self.h)),
                   "rs_net_create")
        self.n = lib().rs_net_num_params()

    def params(self) -> dict:
        out = np.empty(self.n, dtype=np.float32)
        _check(lib().rs_net_get_params(self.h, out.ctypes.data_as(_f32p), self.n), "rs_net_get_params")
        return net_unflatten(out)

    def grads(self) -> dict:
        out = np.empty(self.n, dtype=np.float32)
        _check(lib().rs_net_get_grads(self.h, out.ctypes.data_as(_f32p), self.n), "rs_net_get_grads")
        return net_unflatten(out)

    def zero_grads(self):
        _check(lib().rs_net_zero_grads(self.h), "rs_net_zero_grads")

    def forward(self, grid, r, logk, out):
        nx, ny, nz = grid
        _check(lib().rs_net_forward(self.h, nx, ny, nz, _vp(r.data_ptr()), _vp(logk.data_ptr()),
                                    _vp(out.data_ptr())), "rs_net_forward")

    def accumulate(self, grid, r, logk, e, weight=1.0, want_loss=False):
        nx, ny, nz = grid
        loss = C.c_double(0.0)
        _check(lib().rs_net_accumulate(self.h, nx, ny, nz, _vp(r.data_ptr()), _vp(logk.data_ptr()),
                                       _vp(e.data_ptr()), weight, C.byref(loss) if want_loss else None),
               "rs_net_accumulate")
        return loss.value if want_loss else None

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().rs_net_adam(self.h, lr, beta1, beta2, eps), "rs_net_adam")

    def save(self, path):
        _check(lib().rs_net_save(self.h, path.encode()), "rs_net_save")

    def __del__(self):
        try:
            if self.h and not _finalizing():
                lib().rs_net_destroy(C.byref(self.h))
        except Exception:
            pass


def _solve(fn, A, M, b, x, *args):
    info = SolveInfo()
    st = fn(A.h, M.h if M is not None else None, b.h, x.h, *args, C.byref(info))
    if st not in (OK, NOT_CONVERGED, ERR_BREAKDOWN):
        raise RsError(st, fn.__name__)
    return info.as_dict()


def solve_gmres(A: Mat, M, b: Vec, x: Vec, restart=30, rtol=1e-8, maxit=10000):
    return _solve(lib().rs_solve_gmres, A, M, b, x, restart, rtol, maxit)


def solve_fgmres(A: Mat, M, b: Vec, x: Vec, restart=30, rtol=1e-8, maxit=10000):
    return _solve(lib().rs_solve_fgmres, A, M, b, x, restart, rtol, maxit)


def solve_lgmres(A: Mat, M, b: Vec, x: Vec, restart=30, aug_k=2, rtol=1e-8, maxit=10000):
    return _solve(lib().rs_solve_lgmres, A, M, b, x, restart, aug_k, rtol, maxit)


def solve_bicgstab(A: Mat, M, b: Vec, x: Vec, rtol=1e-8, maxit=10000):
    return _solve(lib().rs_solve_bicgstab, A, M, b, x, rtol, maxit)


def solve_cg(A: Mat, M, b: Vec, x: Vec, rtol=1e-8, maxit=10000):
    return _solve(lib().rs_solve_cg, A, M, b, x, rtol, maxit)


def vec_dot(x: Vec, y: Vec) -> float:
    out = C.c_double()
    _check(lib().rs_vec_dot(x.h, y.h, C.byref(out)), "rs_vec_dot")
    return out.value


def vec_norm2(x: Vec) -> float:
    out = C.c_double()
    _check(lib().rs_vec_norm2(x.h, C.byref(out)), "rs_vec_norm2")
    return out.value


def vec_axpby(a, x: Vec, b, y: Vec):
    _check(lib().rs_vec_axpby(a, x.h, b, y.h), "rs_vec_axpby")


def vec_axpbyz(a, x: Vec, b, y: Vec, z: Vec):
    _check(lib().rs_vec_axpbyz(a, x.h, b, y.h, z.h), "rs_vec_axpbyz")


def vec_set_value(x: Vec, a):
    _check(lib().rs_vec_set_value(x.h, a), "rs_vec_set_value")
