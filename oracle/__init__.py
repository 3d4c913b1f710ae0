"""CPU oracle of the preconditioned Krylov path — TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded FP64 reference implementations of every step of
the path (SpMV, BLAS-1, ILU(0), block ILU(0), triangular solves, quasi-IMPES
CPR, GMRES / FGMRES / BiCGSTAB) in plain C (oracle.c), plus the learned
pressure stage in numpy (convnet.py).  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import this package.  It shares no
code with the CUDA library; inputs come from the seeded generators in
``synth``.

Parity status: every function here is pinned by tests/test_oracle_pins.py
against closed forms, brute force or textbook special cases.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, NOT_CONVERGED, INVALID, ZERO_PIVOT, BREAKDOWN = 0, 1, -1, -3, -4
PC_NONE, PC_ILU0, PC_BILU0, PC_CPR, PC_CALLBACK, PC_RAS, PC_AMG = 0, 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _declare(_lib)
    return _lib


# ----------------------------------------------------------------------------
# ctypes structures (mirrors of the structs in oracle.c)
# ----------------------------------------------------------------------------
_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_f32p = C.POINTER(C.c_float)
APPLY_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, _f64p, _f64p)


class _Mat(C.Structure):
    _fields_ = [("bs", C.c_int32), ("nrows", C.c_int32), ("ptr", _i32p),
                ("col", _i32p), ("val", _f64p)]


class _PC(C.Structure):
    _fields_ = [("type", C.c_int32), ("mixed", C.c_int32),
                ("n", C.c_int32), ("ptr", _i32p), ("col", _i32p),
                ("lu", _f64p), ("lu32", _f32p),
                ("nb", C.c_int32), ("bs", C.c_int32), ("bptr", _i32p), ("bcol", _i32p),
                ("blu", _f64p), ("bdinv", _f64p), ("blu32", _f32p), ("bdinv32", _f32p),
                ("A", C.POINTER(_Mat)), ("w", _f64p),
                ("pstage", APPLY_FN), ("pstage_user", C.c_void_p),
                ("fn", APPLY_FN), ("user", C.c_void_p), ("form", C.c_int32),
                ("ras", C.c_void_p), ("amg", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("status", C.c_int32),
                ("pad", C.c_int32), ("true_rel_res", C.c_double),
                ("implicit_rel_res", C.c_double)]

    def as_dict(self):
        return dict(iters=self.iters, restarts=self.restarts, status=self.status,
                    true_rel_res=self.true_rel_res, implicit_rel_res=self.implicit_rel_res)


def _declare(L):
    mp = C.POINTER(_Mat)
    L.or_spmv.argtypes = [mp, _f64p, _f64p]
    L.or_amxpby.argtypes = [C.c_double, mp, _f64p, C.c_double, _f64p]
    L.or_axpby.argtypes = [C.c_int64, C.c_double, _f64p, C.c_double, _f64p]
    L.or_axpbyz.argtypes = [C.c_int64, C.c_double, _f64p, C.c_double, _f64p, _f64p]
    L.or_dot.argtypes = [C.c_int64, _f64p, _f64p]
    L.or_dot.restype = C.c_double
    L.or_norm2.argtypes = [C.c_int64, _f64p]
    L.or_norm2.restype = C.c_double
    L.or_set.argtypes = [C.c_int64, C.c_double, _f64p]
    L.or_ilu0.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _i32p]
    L.or_ilu0_solve.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.or_ilu0_solve_f32.argtypes = [C.c_int32, _i32p, _i32p, _f32p, _f64p, _f64p]
    L.or_bilu0.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _i32p]
    L.or_bilu0_solve.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.or_bilu0_solve_f32.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, _f32p, _f32p, _f64p, _f64p]
    L.or_qimpes_weights.argtypes = [mp, _f64p]
    L.or_qimpes_app.argtypes = [mp, _f64p, _f64p]
    L.or_qimpes_restrict.argtypes = [C.c_int32, C.c_int32, _f64p, _f64p, _f64p]
    L.or_prolong.argtypes = [C.c_int32, C.c_int32, _f64p, _f64p]
    L.or_pc_apply.argtypes = [C.POINTER(_PC), C.c_int64, _f64p, _f64p]
    L.or_iluk_symbolic.argtypes = [C.c_int32, _i32p, _i32p, C.c_int32, C.POINTER(_i32p), C.POINTER(_i32p)]
    L.or_ras_setup.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, _f64p, C.c_int32, _i32p, C.c_int32, C.c_int32,
                               C.c_int32, C.c_int32, C.c_double, C.POINTER(C.c_void_p), _i32p]
    L.or_ilut.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_int32, C.c_double, C.POINTER(_i32p),
                          C.POINTER(_i32p), C.POINTER(_f64p), _i32p]
    L.or_ras_free.argtypes = [C.c_void_p]
    L.or_ras_apply.argtypes = [C.c_void_p, _f64p, _f64p]
    L.or_ras_sizes.argtypes = [C.c_void_p, _i32p, C.POINTER(C.c_int64)]
    L.or_ras_export.argtypes = [C.c_void_p, _i32p, _i32p, _i32p, _f64p]
    L.free.argtypes = [C.c_void_p]
    L.or_amg_setup.argtypes = [C.c_int32, _i32p, _i32p, _f64p, C.c_double, C.c_int32, C.c_int32, C.c_int32,
                               C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]
    L.or_splitmix64.argtypes = [C.c_uint64]
    L.or_splitmix64.restype = C.c_uint64
    L.or_pmis.argtypes = [C.c_int32, _i32p, _i32p, _i32p, _i32p, _f64p, C.c_char_p]
    L.or_pmis.restype = C.c_int32
    L.or_hgs_sweep.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_int32, C.c_int32, _f64p]
    L.or_amg_free.argtypes = [C.c_void_p]
    L.or_amg_apply.argtypes = [C.c_void_p, _f64p, _f64p]
    L.or_amg_nlevels.argtypes = [C.c_void_p]
    L.or_amg_nlevels.restype = C.c_int32
    L.or_amg_level_sizes.argtypes = [C.c_void_p, C.c_int32, _i32p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.or_amg_level.argtypes = [C.c_void_p, C.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p]
    L.or_amg_cidx.argtypes = [C.c_void_p, C.c_int32, _i32p]
    L.or_orthogonalise.argtypes = [C.c_int64, C.c_int32, _f64p, _f64p, _f64p, C.c_int32]
    L.or_gmres.argtypes = [mp, C.POINTER(_PC), _f64p, _f64p, C.c_int32, C.c_double, C.c_int32,
                           C.c_int32, C.c_int32, C.c_int32, _f64p, C.c_int32, C.POINTER(Info)]
    L.or_bicgstab.argtypes = [mp, C.POINTER(_PC), _f64p, _f64p, C.c_double, C.c_int32,
                              _f64p, C.c_int32, C.POINTER(Info)]
    L.or_cg.argtypes = [mp, C.POINTER(_PC), _f64p, _f64p, C.c_double, C.c_int32,
                        _f64p, C.c_int32, C.POINTER(Info)]
    L.or_lgmres.argtypes = [mp, C.POINTER(_PC), _f64p, _f64p, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                            C.POINTER(Info)]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------------------
# Matrices
# ----------------------------------------------------------------------------
class Mat:
    """CSR (bs=1) or BSR matrix held for the oracle."""

    def __init__(self, ptr, col, val, bs: int = 1):
        self.bs = int(bs)
        self.ptr, self.col, self.val = _i32(ptr), _i32(col), _f64(val)
        self.nrows = self.ptr.shape[0] - 1
        self.n = self.nrows * self.bs
        self.s = _Mat(self.bs, self.nrows, _p(self.ptr, C.c_int32), _p(self.col, C.c_int32),
                      _p(self.val, C.c_double))

    @classmethod
    def csr(cls, m: dict):
        return cls(m["rowptr"], m["col"], m["val"], 1)

    @classmethod
    def bsr(cls, m: dict):
        return cls(m["browptr"], m["bcol"], m["bval"], m["bs"])


def spmv(A: Mat, x):
    x = _f64(x)
    y = np.empty(A.n)
    lib().or_spmv(C.byref(A.s), _p(x, C.c_double), _p(y, C.c_double))
    return y


def amxpby(a, A: Mat, x, b, y):
    x = _f64(x)
    y = _f64(y).copy()
    lib().or_amxpby(a, C.byref(A.s), _p(x, C.c_double), b, _p(y, C.c_double))
    return y


def axpby(a, x, b, y):
    x, y = _f64(x), _f64(y).copy()
    lib().or_axpby(x.size, a, _p(x, C.c_double), b, _p(y, C.c_double))
    return y


def axpbyz(a, x, b, y):
    x, y = _f64(x), _f64(y)
    z = np.empty_like(x)
    lib().or_axpbyz(x.size, a, _p(x, C.c_double), b, _p(y, C.c_double), _p(z, C.c_double))
    return z


def dot(x, y):
    x, y = _f64(x), _f64(y)
    return lib().or_dot(x.size, _p(x, C.c_double), _p(y, C.c_double))


def norm2(x):
    x = _f64(x)
    return lib().or_norm2(x.size, _p(x, C.c_double))


def set_value(n, v):
    x = np.empty(n)
    lib().or_set(n, v, _p(x, C.c_double))
    return x


# ----------------------------------------------------------------------------
# Factorisations and triangular solves
# ----------------------------------------------------------------------------
def ilu0(A: Mat):
    """ILU(0) factors in A's pattern; returns (status, bad_row, lu)."""
    assert A.bs == 1
    lu = np.empty_like(A.val)
    bad = C.c_int32(-1)
    st = lib().or_ilu0(A.nrows, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                       _p(A.val, C.c_double), _p(lu, C.c_double), C.byref(bad))
    return st, bad.value, lu


def ilu0_solve(A: Mat, lu, r, fp32: bool = False):
    r = _f64(r)
    z = np.empty(A.n)
    if fp32:
        lu32 = np.ascontiguousarray(lu, dtype=np.float32)
        lib().or_ilu0_solve_f32(A.nrows, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                                _p(lu32, C.c_float), _p(r, C.c_double), _p(z, C.c_double))
    else:
        lu = _f64(lu)
        lib().or_ilu0_solve(A.nrows, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                            _p(lu, C.c_double), _p(r, C.c_double), _p(z, C.c_double))
    return z


def bilu0(A: Mat):
    """Block ILU(0); returns (status, bad_block_row, lu, dinv)."""
    lu = np.empty_like(A.val)
    dinv = np.empty(A.nrows * A.bs * A.bs)
    bad = C.c_int32(-1)
    st = lib().or_bilu0(A.nrows, A.bs, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                        _p(A.val, C.c_double), _p(lu, C.c_double), _p(dinv, C.c_double),
                        C.byref(bad))
    return st, bad.value, lu, dinv


def bilu0_solve(A: Mat, lu, dinv, r, fp32: bool = False):
    r = _f64(r)
    z = np.empty(A.n)
    if fp32:
        lu32 = np.ascontiguousarray(lu, dtype=np.float32)
        d32 = np.ascontiguousarray(dinv, dtype=np.float32)
        lib().or_bilu0_solve_f32(A.nrows, A.bs, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                                 _p(lu32, C.c_float), _p(d32, C.c_float),
                                 _p(r, C.c_double), _p(z, C.c_double))
    else:
        lib().or_bilu0_solve(A.nrows, A.bs, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                             _p(_f64(lu), C.c_double), _p(_f64(dinv), C.c_double),
                             _p(r, C.c_double), _p(z, C.c_double))
    return z


def qimpes_weights(A: Mat):
    w = np.empty(A.nrows * (A.bs - 1))
    lib().or_qimpes_weights(C.byref(A.s), _p(w, C.c_double))
    return w


def qimpes_app(A: Mat, w):
    w = _f64(w)
    app = np.empty(A.col.shape[0])
    lib().or_qimpes_app(C.byref(A.s), _p(w, C.c_double), _p(app, C.c_double))
    return app


def qimpes_restrict(nb, bs, w, f):
    w, f = _f64(w), _f64(f)
    rp = np.empty(nb)
    lib().or_qimpes_restrict(nb, bs, _p(w, C.c_double), _p(f, C.c_double), _p(rp, C.c_double))
    return rp


def prolong(nb, bs, p):
    p = _f64(p)
    z = np.empty(nb * bs)
    lib().or_prolong(nb, bs, _p(p, C.c_double), _p(z, C.c_double))
    return z


def orthogonalise(V, w, i, mgs=False):
    """CGS2 (or MGS) step against columns 0..i of V (shape (k, n), row k = v_k)."""
    V = _f64(V)
    w = _f64(w).copy()
    n = w.size
    h = np.zeros(i + 2)
    lib().or_orthogonalise(n, i, _p(V, C.c_double), _p(w, C.c_double), _p(h, C.c_double), int(mgs))
    return w, h


def iluk_pattern(n, ptr, col, p):
    """ILU(p) pattern by level of fill: (ptr, col) of the kept entries."""
    ptr, col = _i32(ptr), _i32(col)
    op, oc = _i32p(), _i32p()
    lib().or_iluk_symbolic(n, _p(ptr, C.c_int32), _p(col, C.c_int32), p, C.byref(op), C.byref(oc))
    optr = np.ctypeslib.as_array(op, shape=(n + 1,)).copy()
    ocol = np.ctypeslib.as_array(oc, shape=(max(int(optr[-1]), 1),))[:int(optr[-1])].copy()
    lib().free(C.cast(op, C.c_void_p))
    lib().free(C.cast(oc, C.c_void_p))
    return optr, ocol


def ilut(A: Mat, p: int, tol: float):
    """ILUT(p, tol) of a CSR matrix: (status, bad_row, ptr, col, lu) in the
    factor's own pattern (strict L, then U with its diagonal)."""
    assert A.bs == 1
    op, oc, ov = _i32p(), _i32p(), _f64p()
    bad = C.c_int32(-1)
    st = lib().or_ilut(A.nrows, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32), _p(A.val, C.c_double), p, tol,
                       C.byref(op), C.byref(oc), C.byref(ov), C.byref(bad))
    if st != OK:
        return st, bad.value, None, None, None
    n = A.nrows
    ptr = np.ctypeslib.as_array(op, shape=(n + 1,)).copy()
    nz = int(ptr[-1])
    col = np.ctypeslib.as_array(oc, shape=(max(nz, 1),))[:nz].copy()
    lu = np.ctypeslib.as_array(ov, shape=(max(nz, 1),))[:nz].copy()
    for q in (op, oc, ov):
        lib().free(C.cast(q, C.c_void_p))
    return st, bad.value, ptr, col, lu


def contiguous_partition(n, nsub):
    """Row i -> subdomain floor(i nsub / n): contiguous blocks of rows, the
    way the paper's MAP gives each process a range of rows."""
    return (np.arange(n, dtype=np.int64) * nsub // max(n, 1)).astype(np.int32)


class Ras:
    """Restricted additive Schwarz with ILU(level) local solvers; on a block
    matrix the subdomains hold block rows and the local solver is block ILU."""

    def __init__(self, A: Mat, nsub: int, part=None, overlap: int = 1, level: int = 0, ilut=None):
        """ilut = (p, tol) selects ILUT(p, tol) local solvers instead of ILU(level)."""
        self.A = A
        self.part = _i32(contiguous_partition(A.nrows, nsub) if part is None else part)
        h = C.c_void_p()
        bad = C.c_int32(-1)
        p, tol = ilut if ilut is not None else (0, 0.0)
        self.status = lib().or_ras_setup(A.nrows, A.bs, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                                         _p(A.val, C.c_double), nsub, _p(self.part, C.c_int32), overlap,
                                         level, 1 if ilut is not None else 0, p, tol, C.byref(h), C.byref(bad))
        self.bad = bad.value
        self.h = h

    def apply(self, r):
        r = _f64(r)
        z = np.empty_like(r)
        lib().or_ras_apply(self.h, _p(r, C.c_double), _p(z, C.c_double))
        return z

    def structure(self):
        """The stacked block-diagonal local problems: (gidx, ptr, col, lu)."""
        ne = C.c_int32()
        nz = C.c_int64()
        lib().or_ras_sizes(self.h, C.byref(ne), C.byref(nz))
        gidx = np.empty(ne.value, np.int32)
        ptr = np.empty(ne.value + 1, np.int32)
        col = np.empty(nz.value, np.int32)
        lu = np.empty(nz.value * self.A.bs * self.A.bs)
        lib().or_ras_export(self.h, _p(gidx, C.c_int32), _p(ptr, C.c_int32), _p(col, C.c_int32),
                            _p(lu, C.c_double))
        return gidx, ptr, col, lu

    def __del__(self):
        try:
            if self.h:
                lib().or_ras_free(self.h)
        except Exception:
            pass


def hgs_sweep(A: Mat, b, x, chunk=32, backward=False):
    """One hybrid Gauss-Seidel sweep (Fig. 34's relaxation): Gauss-Seidel in
    row order (backward: reverse order) inside chunks of `chunk` consecutive
    rows, Jacobi between chunks.  Returns (status, new x)."""
    assert A.bs == 1
    b, x = _f64(b), _f64(x)
    out = np.empty_like(x)
    st = lib().or_hgs_sweep(A.nrows, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32), _p(A.val, C.c_double),
                            _p(b, C.c_double), _p(x, C.c_double), chunk, int(backward), _p(out, C.c_double))
    return st, out


def splitmix64(k):
    """The k-th output of SplitMix64 from state 0 (the PMIS weights' generator)."""
    return int(lib().or_splitmix64(k))


def pmis(n, sptr, scol, w):
    """PMIS C/F splitting (Sec. 4.2's PMIS) of the strength graph S (sptr,
    scol: the points each point strongly depends on) with weights w: returns
    (states, rounds), states 1 for C and 2 for F."""
    sptr, scol, w = np.ascontiguousarray(sptr, np.int32), np.ascontiguousarray(scol, np.int32), _f64(w)
    # S^T by counting, rows in order
    tptr = np.zeros(n + 1, np.int32)
    np.add.at(tptr, scol + 1, 1)
    tptr = np.cumsum(tptr).astype(np.int32)
    tcol = np.empty(scol.size, np.int32)
    fill = tptr[:-1].copy()
    for i in range(n):
        for q in range(sptr[i], sptr[i + 1]):
            tcol[fill[scol[q]]] = i
            fill[scol[q]] += 1
    st = C.create_string_buffer(max(n, 1))
    rounds = lib().or_pmis(n, _p(sptr, C.c_int32), _p(scol, C.c_int32), _p(tptr, C.c_int32), _p(tcol, C.c_int32),
                           _p(w, C.c_double), st)
    return np.frombuffer(st.raw[:n], np.int8).astype(np.int32), rounds


class Amg:
    """Algebraic multigrid V-cycle (Algs. 3-4): classical strength (theta),
    coarsening by PMIS (default; weights from SplitMix64 keyed by level and
    point) or the Ruge-Stueben first pass (coarsen="rs"), direct
    interpolation, Galerkin coarse matrices, nu smoothing sweeps before and
    after (smoother 0: l1-Jacobi; 1: hybrid Gauss-Seidel over 32-row chunks,
    forward before and backward after the coarse correction), dense coarsest
    solve."""

    def __init__(self, A: Mat, theta=0.5, max_levels=16, max_coarse=256, nu=2, smoother=0, coarsen="pmis"):
        assert A.bs == 1
        self.A = A
        h = C.c_void_p()
        self.status = lib().or_amg_setup(A.nrows, _p(A.ptr, C.c_int32), _p(A.col, C.c_int32),
                                         _p(A.val, C.c_double), theta, max_levels, max_coarse, nu, smoother,
                                         {"rs": 0, "pmis": 1}[coarsen], C.byref(h))
        self.h = h

    def apply(self, r):
        r = _f64(r)
        z = np.empty_like(r)
        lib().or_amg_apply(self.h, _p(r, C.c_double), _p(z, C.c_double))
        return z

    def cidx(self, l=0):
        """Coarse index of every point of level l (-1 for F points)."""
        n = self.levels()[l][0][0].size - 1
        out = np.empty(n, np.int32)
        lib().or_amg_cidx(self.h, l, _p(out, C.c_int32))
        return out

    def levels(self):
        """[(A_l as (ptr, col, val), P_l as (ptr, col, val) or None)] per level."""
        out = []
        L = lib()
        nl = L.or_amg_nlevels(self.h)
        for l in range(nl):
            n, na, np_ = C.c_int32(), C.c_int64(), C.c_int64()
            L.or_amg_level_sizes(self.h, l, C.byref(n), C.byref(na), C.byref(np_))
            a = (np.empty(n.value + 1, np.int32), np.empty(na.value, np.int32), np.empty(na.value))
            p = (np.empty(n.value + 1, np.int32), np.empty(np_.value, np.int32), np.empty(np_.value)) \
                if l + 1 < nl else None
            L.or_amg_level(self.h, l, _p(a[0], C.c_int32), _p(a[1], C.c_int32), _p(a[2], C.c_double),
                           _p(p[0], C.c_int32) if p else None, _p(p[1], C.c_int32) if p else None,
                           _p(p[2], C.c_double) if p else None)
            out.append((a, p))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().or_amg_free(self.h)
        except Exception:
            pass


# ----------------------------------------------------------------------------
# Preconditioners
# ----------------------------------------------------------------------------
class PC:
    """Oracle preconditioner: none / ilu0 / bilu0 / cpr / callback / ras.

    kind='ras': restricted additive Schwarz, `ras` = dict(nsub=, part=,
    overlap=, level=) as for Ras.
    kind='amg': one AMG V-cycle, `amg` = keyword arguments of Amg; with
    kind='cpr', `amg` makes the pressure stage one AMG V-cycle on App' and
    `ras` makes the F stage restricted additive Schwarz on A.

    kind='cpr' on a BSR matrix: quasi-IMPES restriction, ILU(0) of App'
    (or `pstage`, a callable rp -> zp), prolongation, residual, block ILU(0).
    kind='cpr' on a CSR matrix (bs=1): restriction = identity, App' = A,
    second stage = ILU(0) of A.
    form: the order of the stages (F = block ILU(0) of A, P = pressure
    stage): 'pf' (Alg. 6 as read), 'fp' (Alg. 5), 'fpf' (Alg. 7), 'ffpf'
    (Alg. 8).
    """

    FORMS = ("pf", "fp", "fpf", "ffpf")   # Algs. 6, 5, 7, 8

    def __init__(self, A: Mat, kind: str = "ilu0", mixed: bool = False, pstage=None, fn=None, form: str = "pf",
                 ras=None, amg=None):
        self.A = A
        self.kind = kind
        self._keep = []
        s = _PC()
        s.mixed = int(mixed)
        s.form = self.FORMS.index(form)
        self.status = OK
        if kind == "none":
            s.type = PC_NONE
        elif kind == "ilu0":
            st, bad, lu = ilu0(A)
            self.status, self.bad = st, bad
            self.lu = lu
            self._set_ilu(s, A.ptr, A.col, A.nrows, lu)
            s.type = PC_ILU0
        elif kind == "bilu0":
            self._set_bilu(s, A)
            s.type = PC_BILU0
        elif kind == "cpr":
            self._set_bilu(s, A)
            if A.bs > 1:
                self.w = qimpes_weights(A)
                self.app_val = qimpes_app(A, self.w)
            else:
                self.w = np.zeros(0)
                self.app_val = A.val.copy()
            self.App = Mat(A.ptr, A.col, self.app_val, 1)
            if ras is not None:                     # RAS as the F stage R(A)^{-1} (Sec. 4.2.1)
                self.fras = Ras(A, **ras)
                if self.fras.status != OK:
                    self.status = self.fras.status
                s.ras = self.fras.h
            if amg is not None:                     # AMG V-cycle pressure stage (Sec. 4.2)
                self.amg = Amg(self.App, **amg)
                if self.amg.status != OK:
                    self.status = self.amg.status
                s.amg = self.amg.h
            st, bad, lu = ilu0(self.App)
            if st != OK:
                self.status, self.bad = st, bad
            self.lu = lu
            self._set_ilu(s, A.ptr, A.col, A.nrows, lu)
            s.A = C.pointer(A.s)
            s.w = _p(self.w, C.c_double) if self.w.size else None
            if pstage is not None:
                s.pstage = self._wrap(pstage)
            s.type = PC_CPR
        elif kind == "callback":
            s.fn = self._wrap(fn)
            s.type = PC_CALLBACK
        elif kind == "ras":
            self.ras = Ras(A, **(ras or {}))
            self.status, self.bad = self.ras.status, self.ras.bad
            s.ras = self.ras.h
            s.type = PC_RAS
        elif kind == "amg":
            self.amg = Amg(A, **(amg or {}))
            self.status = self.amg.status
            s.amg = self.amg.h
            s.type = PC_AMG
        else:
            raise ValueError(kind)
        self.s = s

    def _wrap(self, f):
        def cb(user, n, r, z):
            rv = np.ctypeslib.as_array(r, shape=(n,))
            zv = np.ctypeslib.as_array(z, shape=(n,))
            zv[:] = f(rv.copy())
            return 0
        cfn = APPLY_FN(cb)
        self._keep.append(cfn)
        return cfn

    def _set_ilu(self, s, ptr, col, n, lu):
        self.lu32 = lu.astype(np.float32)
        self._keep += [ptr, col, lu, self.lu32]
        s.n = n
        s.ptr, s.col = _p(ptr, C.c_int32), _p(col, C.c_int32)
        s.lu, s.lu32 = _p(lu, C.c_double), _p(self.lu32, C.c_float)

    def _set_bilu(self, s, A):
        st, bad, blu, dinv = bilu0(A)
        self.bstatus = st
        if st != OK:
            self.status, self.bad = st, bad
        self.blu, self.bdinv = blu, dinv
        self.blu32, self.bdinv32 = blu.astype(np.float32), dinv.astype(np.float32)
        self._keep += [blu, dinv, self.blu32, self.bdinv32]
        s.nb, s.bs = A.nrows, A.bs
        s.bptr, s.bcol = _p(A.ptr, C.c_int32), _p(A.col, C.c_int32)
        s.blu, s.bdinv = _p(blu, C.c_double), _p(dinv, C.c_double)
        s.blu32, s.bdinv32 = _p(self.blu32, C.c_float), _p(self.bdinv32, C.c_float)

    def apply(self, r):
        r = _f64(r)
        z = np.empty_like(r)
        st = lib().or_pc_apply(C.byref(self.s), r.size, _p(r, C.c_double), _p(z, C.c_double))
        if st != OK:
            raise RuntimeError("oracle preconditioner apply failed: %d" % st)
        return z


# ----------------------------------------------------------------------------
# Solvers
# ----------------------------------------------------------------------------
def gmres(A: Mat, M: PC | None, b, x0=None, restart=30, rtol=1e-8, maxit=10000,
          side="right", flexible=False, mgs=False, hist_len=0):
    """Restarted GMRES(m) / FGMRES(m); returns (x, info dict, history)."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    info = Info()
    hist = np.zeros(max(hist_len, 1))
    Ms = M.s if M is not None else PC(A, "none").s
    lib().or_gmres(C.byref(A.s), C.byref(Ms), _p(b, C.c_double), _p(x, C.c_double),
                   restart, rtol, maxit, 1 if side == "left" else 0, int(flexible), int(mgs),
                   _p(hist, C.c_double), hist_len, C.byref(info))
    return x, info.as_dict(), hist[:min(hist_len, info.iters)]


def fgmres(A, M, b, x0=None, restart=30, rtol=1e-8, maxit=10000, hist_len=0):
    return gmres(A, M, b, x0, restart, rtol, maxit, "right", True, False, hist_len)


def lgmres(A: Mat, M: PC | None, b, x0=None, restart=30, aug_k=2, rtol=1e-8, maxit=10000):
    """LGMRES(restart, aug_k): flexible GMRES augmented with the last aug_k
    normalised corrections.  Returns (x, info)."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    info = Info()
    pc = M.s if M is not None else PC(A, "none").s
    lib().or_lgmres(C.byref(A.s), C.byref(pc), _p(b, C.c_double), _p(x, C.c_double), restart, aug_k, rtol,
                    maxit, C.byref(info))
    return x, info.as_dict()


def cg(A: Mat, M: PC | None, b, x0=None, rtol=1e-8, maxit=10000, hist_len=0):
    """Preconditioned conjugate gradient (Alg. 2) for SPD A and M."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    info = Info()
    hist = np.zeros(max(hist_len, 1))
    Ms = M.s if M is not None else PC(A, "none").s
    lib().or_cg(C.byref(A.s), C.byref(Ms), _p(b, C.c_double), _p(x, C.c_double),
                rtol, maxit, _p(hist, C.c_double), hist_len, C.byref(info))
    return x, info.as_dict(), hist[:min(hist_len, info.iters)]


def bicgstab(A: Mat, M: PC | None, b, x0=None, rtol=1e-8, maxit=10000, hist_len=0):
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    info = Info()
    hist = np.zeros(max(hist_len, 1))
    Ms = M.s if M is not None else PC(A, "none").s
    lib().or_bicgstab(C.byref(A.s), C.byref(Ms), _p(b, C.c_double), _p(x, C.c_double),
                      rtol, maxit, _p(hist, C.c_double), hist_len, C.byref(info))
    return x, info.as_dict(), hist[:min(hist_len, info.iters)]
