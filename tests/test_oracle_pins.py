"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks one oracle function against a closed form, brute force on a
tiny input, a textbook special case or an algebraic invariant, chosen so that
a dropped term, a wrong sign, a wrong index or a transposed operand fails.
CPU only.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers building small test matrices (inputs only)
# ----------------------------------------------------------------------------
def csr_dict(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return dict(n=A.shape[0], rowptr=A.indptr.astype(np.int32), col=A.indices.astype(np.int32),
                val=A.data.astype(np.float64))


def dense_pattern_csr(D):
    """Every entry of a dense matrix stored explicitly (a full pattern)."""
    n = D.shape[0]
    return dict(n=n, rowptr=(np.arange(n + 1) * n).astype(np.int32),
                col=np.tile(np.arange(n), n).astype(np.int32), val=D.reshape(-1).copy())


def poisson1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def poisson3d_dirichlet(nx, ny, nz):
    Ix, Iy, Iz = sp.eye(nx), sp.eye(ny), sp.eye(nz)
    return (sp.kron(Iz, sp.kron(Iy, poisson1d(nx))) + sp.kron(Iz, sp.kron(poisson1d(ny), Ix))
            + sp.kron(poisson1d(nz), sp.kron(Iy, Ix))).tocsr()


def eig1d(n, k):
    j = np.arange(1, n + 1)
    return np.sin(k * np.pi * j / (n + 1)), 2.0 - 2.0 * np.cos(k * np.pi / (n + 1))


def lu_dense_from_ilu(d, lu):
    """Dense L (unit lower) and U from factors stored in d's pattern."""
    n = d["n"]
    L, U = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for p in range(d["rowptr"][i], d["rowptr"][i + 1]):
            j = d["col"][p]
            if j < i:
                L[i, j] = lu[p]
            else:
                U[i, j] = lu[p]
    return L, U


# ----------------------------------------------------------------------------
# generator (inputs)
# ----------------------------------------------------------------------------
def test_generator_pressure_matrix_properties():
    g = synth.Grid(6, 5, 4)
    m = synth.pressure_7pt(g, 7, kz_scale=0.1)
    A = sp.csr_matrix((m["val"], m["col"], m["rowptr"]), shape=(g.n, g.n)).toarray()
    assert np.allclose(A, A.T, rtol=0, atol=0)
    assert np.allclose(A.sum(axis=1), 1e-3, rtol=0, atol=1e-12)
    off = A - np.diag(np.diag(A))
    assert (off <= 0).all() and (np.diag(A) > 0).all()
    nnz = 7 * g.n - 2 * (g.nx * g.ny + g.ny * g.nz + g.nx * g.nz)
    assert m["col"].size == nnz
    for i in range(g.n):
        c = m["col"][m["rowptr"][i]:m["rowptr"][i + 1]]
        assert (np.diff(c) > 0).all() and i in c
    m2 = synth.pressure_7pt(g, 7, kz_scale=0.1)
    m3 = synth.pressure_7pt(g, 8, kz_scale=0.1)
    assert np.array_equal(m["val"], m2["val"]) and not np.array_equal(m["val"], m3["val"])


def test_generator_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first three
    outputs of the published generator are 0xE220A8397B1DCDAF,
    0x6E789E6AA1B965F4 and 0x06C45D188009454F (state advanced by the
    golden gamma 0x9E3779B97F4A7C15 before each output)."""
    gamma = 0x9E3779B97F4A7C15
    states = np.array([0, gamma, (2 * gamma) % 2 ** 64], dtype=np.uint64)
    out = [int(v) for v in synth.splitmix64(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_generator_determinism_pin():
    """The generator's output is the committed one (tests/golden/synth_pin.txt,
    written by make_synth_pin.py): patterns by SHA-256, values within 1e-13."""
    import hashlib
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_synth_pin", os.path.join(GOLDEN, "make_synth_pin.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    pinned = {}
    for line in open(os.path.join(GOLDEN, "synth_pin.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, key, kind, rest = line.split(" ", 3)
        pinned[(name, key)] = (kind, rest.split())
    seen = 0
    for name, d in mk.cases():
        for key in sorted(d):
            a = np.asarray(d[key])
            if (name, key) not in pinned:
                continue
            kind, rest = pinned[(name, key)]
            if kind == "sha256":
                assert hashlib.sha256(a.astype("<i4").tobytes()).hexdigest() == rest[0], (name, key)
            else:
                ref = np.array([float(v) for v in rest])
                assert a.shape == ref.shape and np.allclose(a, ref, rtol=1e-13, atol=0), (name, key)
            seen += 1
    assert seen == len(pinned) and seen >= 19


def test_generator_bsr_properties():
    g = synth.Grid(4, 3, 3)
    m = synth.black_oil_bsr3(g, 3)
    c = synth.csr_from_bsr(m)
    A = sp.csr_matrix((c["val"], c["col"], c["rowptr"]), shape=(c["n"], c["n"])).toarray()
    p = synth.pressure_7pt(g, 3)
    App = sp.csr_matrix((p["val"], p["col"], p["rowptr"]), shape=(g.n, g.n)).toarray()
    assert np.array_equal(A[0::3, 0::3], App)
    for s in (1, 2):
        rows = A[s::3]
        d = np.abs(rows[np.arange(g.n), np.arange(g.n) * 3 + s])
        others = np.abs(rows).sum(axis=1) - d
        assert (d > others).all()                       # diagonally dominant saturation rows
        assert np.allclose(A[s::3, 0::3].sum(axis=1), 0, atol=1e-12)  # zero-sum pressure part


# ----------------------------------------------------------------------------
# SpMV and BLAS-1 (Sec. 2.2-2.3, Figs. 10-13, 20-21)
# ----------------------------------------------------------------------------
def test_spmv_integer_exact(orc):
    rng = np.random.default_rng(0)
    n = 57
    D = rng.integers(-5, 6, size=(n, n)).astype(float)
    D[rng.random((n, n)) < 0.8] = 0.0
    D[3, :] = 0.0                                       # an empty row
    d = csr_dict(D)
    x = rng.integers(-9, 10, size=n).astype(float)
    A = orc.Mat.csr(d)
    assert np.array_equal(orc.spmv(A, x), D @ x)
    y = rng.integers(-9, 10, size=n).astype(float)
    assert np.array_equal(orc.amxpby(2.0, A, x, -3.0, y), 2.0 * (D @ x) - 3.0 * y)


def test_bsr_spmv_integer_exact(orc):
    rng = np.random.default_rng(1)
    nb, bs = 11, 3
    mask = rng.random((nb, nb)) < 0.35
    np.fill_diagonal(mask, True)
    ptr = np.concatenate([[0], np.cumsum(mask.sum(axis=1))]).astype(np.int32)
    col = np.nonzero(mask)[1].astype(np.int32)
    blocks = rng.integers(-4, 5, size=(col.size, bs, bs)).astype(float)
    D = np.zeros((nb * bs, nb * bs))
    k = 0
    for I in range(nb):
        for J in np.nonzero(mask[I])[0]:
            D[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = blocks[k]
            k += 1
    A = orc.Mat(ptr, col, blocks.reshape(-1), bs)
    x = rng.integers(-9, 10, size=nb * bs).astype(float)
    assert np.array_equal(orc.spmv(A, x), D @ x)
    y = np.arange(nb * bs, dtype=float)
    assert np.array_equal(orc.amxpby(-1.0, A, x, 1.0, y), y - D @ x)


def test_blas1_closed_forms(orc):
    n = 1000
    x = np.arange(1, n + 1, dtype=float)
    assert orc.dot(x, x) == n * (n + 1) * (2 * n + 1) / 6
    assert orc.norm2(np.ones(n)) == np.sqrt(n)
    y = x[::-1].copy()                                   # n+1-i
    assert np.array_equal(orc.axpby(2.0, x, 3.0, y), 2 * x + 3 * (n + 1 - x))
    assert np.array_equal(orc.axpbyz(-1.0, x, 1.0, y, ), (n + 1) - 2 * x)
    assert np.array_equal(orc.set_value(5, 2.5), np.full(5, 2.5))
    assert orc.dot(x, -x) == -orc.dot(x, x)


# ----------------------------------------------------------------------------
# ILU(0) and triangular solves (Sec. 4.1, Eq. 3)
# ----------------------------------------------------------------------------
def test_ilu0_tridiagonal_is_exact_lu(orc):
    rng = np.random.default_rng(2)
    n = 40
    D = np.diag(3 + rng.random(n)) + np.diag(-rng.random(n - 1), 1) + np.diag(-rng.random(n - 1), -1)
    d = csr_dict(D)
    st, bad, lu = orc.ilu0(orc.Mat.csr(d))
    assert st == 0
    L, U = lu_dense_from_ilu(d, lu)
    P, Lr, Ur = sla.lu(D)
    assert np.array_equal(P, np.eye(n))                 # no pivoting needed: plain LU
    assert np.allclose(L, Lr, rtol=0, atol=1e-14) and np.allclose(U, Ur, rtol=1e-14, atol=1e-14)


def test_ilu0_dense_pattern_is_lu(orc):
    rng = np.random.default_rng(3)
    n = 12
    D = rng.standard_normal((n, n)) + n * np.eye(n)
    d = dense_pattern_csr(D)
    st, _, lu = orc.ilu0(orc.Mat.csr(d))
    assert st == 0
    L, U = lu_dense_from_ilu(d, lu)
    P, Lr, Ur = sla.lu(D)
    if np.array_equal(P, np.eye(n)):
        assert np.allclose(L, Lr, atol=1e-13) and np.allclose(U, Ur, atol=1e-12)
    assert np.allclose(L @ U, D, atol=1e-12)


def test_ilu0_pattern_invariant_7pt(orc):
    g = synth.Grid(5, 4, 3)
    d = synth.pressure_7pt(g, 11)
    st, _, lu = orc.ilu0(orc.Mat.csr(d))
    assert st == 0
    L, U = lu_dense_from_ilu(d, lu)
    A = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(g.n, g.n)).toarray()
    P = A != 0
    LU = L @ U
    assert np.allclose(LU[P], A[P], rtol=1e-13, atol=1e-13)     # (LU)_ij = a_ij on pat(A)
    assert np.abs(LU[~P]).max() > 1e-6                           # fill was dropped (not exact LU)
    assert (np.tril(L, -1)[~P] == 0).all() and (U[~P] == 0).all()


def test_ilu0_zero_pivot_reported(orc):
    D = np.array([[1.0, 2.0, 0.0], [0.5, 1.0, 1.0], [0.0, 1.0, 3.0]])   # u_11 = 1 - 0.5*2 = 0
    st, bad, _ = orc.ilu0(orc.Mat.csr(csr_dict(D)))
    assert st == orc.ZERO_PIVOT and bad == 1


def test_ilu0_solve_tridiagonal_is_thomas(orc):
    rng = np.random.default_rng(4)
    n = 64
    lo, dg, up = -rng.random(n - 1), 3 + rng.random(n), -rng.random(n - 1)
    D = np.diag(dg) + np.diag(up, 1) + np.diag(lo, -1)
    d = csr_dict(D)
    A = orc.Mat.csr(d)
    _, _, lu = orc.ilu0(A)
    r = rng.standard_normal(n)
    ab = np.zeros((3, n))
    ab[0, 1:], ab[1], ab[2, :-1] = up, dg, lo
    z_ref = sla.solve_banded((1, 1), ab, r)
    assert np.allclose(orc.ilu0_solve(A, lu, r), z_ref, rtol=1e-13, atol=1e-13)


def test_ilu0_solve_inverts_lu(orc):
    g = synth.Grid(6, 5, 4)
    d = synth.pressure_7pt(g, 5, kz_scale=0.1)
    A = orc.Mat.csr(d)
    _, _, lu = orc.ilu0(A)
    L, U = lu_dense_from_ilu(d, lu)
    r = np.random.default_rng(5).standard_normal(g.n)
    z = orc.ilu0_solve(A, lu, r)
    assert np.linalg.norm(L @ (U @ z) - r) <= 1e-13 * np.linalg.norm(r)
    z32 = orc.ilu0_solve(A, lu, r, fp32=True)
    assert np.linalg.norm(z32 - z) <= 1e-5 * np.linalg.norm(z)
    assert np.linalg.norm(z32 - z) > 0


def _read_golden_kv(name):
    """key = values lines of a golden file (values as hex or decimal floats)."""
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0]
        if "=" not in line:
            continue
        k, v = line.split("=", 1)
        out[k.strip()] = [float.fromhex(t) if "x" in t else float(t) for t in v.split()]
    return out


def test_ilu0_solve_f32_golden(orc):
    """The FP32 ILU(0) solve against a four-row example worked by hand
    (tests/golden/ilu0_solve_f32_four_rows.txt): every product and every
    difference rounded to binary32.  The example is built so that the
    plausible slips give other bits: an FP64 accumulator with FP32 factors
    (a tie in the product of row 1 goes the other way, and that changes
    rows 0 and 3 too), or one rounding per row (row 3)."""
    g = _read_golden_kv("ilu0_solve_f32_four_rows.txt")
    n = int(g["n"][0])
    A = orc.Mat(np.array(g["rowptr"], np.int32), np.array(g["col"], np.int32), np.zeros(len(g["col"])), 1)
    lu = np.array(g["lu"], np.float32)
    assert np.array_equal(lu.astype(np.float64), np.array(g["lu"]))   # the factors are binary32 values
    r = np.array(g["r"])
    z = orc.ilu0_solve(A, lu, r, fp32=True)
    assert z.shape == (n,) and np.array_equal(z, np.array(g["z"])), (z, g["z"])
    # the FP64 solve with the same factors, rounded to binary32 at the end,
    # differs in every row but row 2
    z64 = orc.ilu0_solve(A, lu.astype(np.float64), r).astype(np.float32).astype(np.float64)
    assert [bool(a != b) for a, b in zip(z64, g["z"])] == [True, True, False, True], z64


def test_bilu0_solve_f32_golden(orc):
    """The FP32 block ILU(0) solve (2x2 blocks) against an example worked by
    hand (tests/golden/bilu0_solve_f32_three_blocks.txt); an FP64 accumulator
    or one rounding per row gives other bits."""
    g = _read_golden_kv("bilu0_solve_f32_three_blocks.txt")
    nb, bs = int(g["nb"][0]), int(g["bs"][0])
    A = orc.Mat(np.array(g["browptr"], np.int32), np.array(g["bcol"], np.int32),
                np.zeros(len(g["bcol"]) * bs * bs), bs)
    lu, dinv = np.array(g["lu"], np.float32), np.array(g["dinv"], np.float32)
    r = np.array(g["r"])
    z = orc.bilu0_solve(A, lu, dinv, r, fp32=True)
    assert z.shape == (nb * bs,) and np.array_equal(z, np.array(g["z"])), (z, g["z"])
    z64 = orc.bilu0_solve(A, lu.astype(np.float64), dinv.astype(np.float64), r)
    z64 = z64.astype(np.float32).astype(np.float64)
    assert [bool(a != b) for a, b in zip(z64, g["z"])] == [False, False, True, False, True, True], z64


# ----------------------------------------------------------------------------
# Block ILU(0)
# ----------------------------------------------------------------------------
def _block_dense(m):
    c = synth.csr_from_bsr(m)
    return sp.csr_matrix((c["val"], c["col"], c["rowptr"]), shape=(c["n"], c["n"])).toarray()


def _block_lu_dense(m, lu, dinv):
    nb, bs = m["nb"], m["bs"]
    L, U = np.eye(nb * bs), np.zeros((nb * bs, nb * bs))
    blk = lu.reshape(-1, bs, bs)
    for I in range(nb):
        for p in range(m["browptr"][I], m["browptr"][I + 1]):
            J = m["bcol"][p]
            tgt = L if J < I else U
            tgt[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = blk[p]
    return L, U


def test_bilu0_bs1_equals_ilu0(orc):
    d = synth.pressure_7pt(synth.Grid(5, 4, 3), 12)
    A = orc.Mat.csr(d)
    _, _, lu = orc.ilu0(A)
    st, _, blu, dinv = orc.bilu0(A)
    assert st == 0
    assert np.allclose(blu, lu, rtol=1e-14, atol=1e-15)
    diag = lu[[np.nonzero(d["col"][d["rowptr"][i]:d["rowptr"][i + 1]] == i)[0][0] + d["rowptr"][i]
               for i in range(d["n"])]]
    assert np.allclose(dinv, 1.0 / diag, rtol=1e-15)


def test_bilu0_block_tridiagonal_is_exact_block_lu(orc):
    m = synth.black_oil_bsr3(synth.Grid(9, 1, 1), 4)     # a 1-D chain: block tridiagonal
    A = orc.Mat.bsr(m)
    st, _, lu, dinv = orc.bilu0(A)
    assert st == 0
    L, U = _block_lu_dense(m, lu, dinv)
    D = _block_dense(m)
    assert np.allclose(L @ U, D, rtol=1e-13, atol=1e-13)
    for I in range(m["nb"]):
        UII = U[3 * I:3 * I + 3, 3 * I:3 * I + 3]
        assert np.allclose(dinv.reshape(-1, 3, 3)[I] @ UII, np.eye(3), atol=1e-13)


def test_bilu0_decoupled_equals_scalar_ilu0(orc):
    """Diagonal blocks only (no coupling between components): block ILU(0)
    splits into three independent scalar ILU(0) factorisations."""
    g = synth.Grid(4, 4, 3)
    ds = [synth.pressure_7pt(g, 20 + s) for s in range(3)]
    ptr, col = ds[0]["rowptr"], ds[0]["col"]
    blocks = np.zeros((col.size, 3, 3))
    for s in range(3):
        blocks[:, s, s] = ds[s]["val"]
    A = orc.Mat(ptr, col, blocks.reshape(-1), 3)
    st, _, lu, dinv = orc.bilu0(A)
    assert st == 0
    lu = lu.reshape(-1, 3, 3)
    for s in range(3):
        _, _, lus = orc.ilu0(orc.Mat.csr(ds[s]))
        assert np.allclose(lu[:, s, s], lus, rtol=1e-14, atol=1e-15)
    off = lu.copy()
    for s in range(3):
        off[:, s, s] = 0
    assert (off == 0).all()


def test_bilu0_solve_inverts_block_lu(orc):
    m = synth.black_oil_bsr3(synth.Grid(4, 3, 3), 6)
    A = orc.Mat.bsr(m)
    st, _, lu, dinv = orc.bilu0(A)
    assert st == 0
    L, U = _block_lu_dense(m, lu, dinv)
    r = np.random.default_rng(6).standard_normal(A.n)
    z = orc.bilu0_solve(A, lu, dinv, r)
    assert np.linalg.norm(L @ (U @ z) - r) <= 1e-12 * np.linalg.norm(r)
    z32 = orc.bilu0_solve(A, lu, dinv, r, fp32=True)
    assert np.linalg.norm(z32 - z) <= 1e-5 * np.linalg.norm(z)


# ----------------------------------------------------------------------------
# Quasi-IMPES CPR (Sec. 4.3, Eqs. 5-9, Alg. 6)
# ----------------------------------------------------------------------------
def _read_golden_qimpes():
    rows = {}
    W = []
    for line in open(os.path.join(GOLDEN, "qimpes_two_cell.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "W":
            W.append([float(v) for v in line[2:]])
        else:
            rows[line[0]] = np.array([float(v) for v in line[1:]])
    return rows, np.array(W)


def test_qimpes_two_cell_golden(orc):
    g, W = _read_golden_qimpes()
    ptr = np.array([0, 2, 4], np.int32)
    col = np.array([0, 1, 0, 1], np.int32)
    val = np.concatenate([g["A00"], g["A01"], g["A10"], g["A11"]])
    A = orc.Mat(ptr, col, val, 3)
    w = orc.qimpes_weights(A)
    assert np.allclose(w.reshape(2, 2), W, rtol=0, atol=1e-15)
    assert np.allclose(orc.qimpes_app(A, w), g["APP"], rtol=0, atol=1e-14)
    assert np.allclose(orc.qimpes_restrict(2, 3, w, g["F"]), g["RP"], rtol=0, atol=1e-14)


def test_restrict_prolong_identity_and_scaling_invariance(orc):
    m = synth.black_oil_bsr3(synth.Grid(4, 3, 2), 9)
    A = orc.Mat.bsr(m)
    w = orc.qimpes_weights(A)
    p = np.random.default_rng(7).standard_normal(m["nb"])
    assert np.array_equal(orc.qimpes_restrict(m["nb"], 3, w, orc.prolong(m["nb"], 3, p)), p)
    # scaling the saturation equations of each cell leaves App' and Pi_r f unchanged
    s = 0.5 + np.random.default_rng(8).random((m["nb"], 2))
    bv = m["bval"].reshape(-1, 3, 3).copy()
    row_of = np.repeat(np.arange(m["nb"]), np.diff(m["browptr"]))
    bv[:, 1, :] *= s[row_of, 0:1]
    bv[:, 2, :] *= s[row_of, 1:2]
    A2 = orc.Mat(m["browptr"], m["bcol"], bv.reshape(-1), 3)
    w2 = orc.qimpes_weights(A2)
    assert np.allclose(orc.qimpes_app(A2, w2), orc.qimpes_app(A, w), rtol=1e-14, atol=1e-14)
    f = np.random.default_rng(9).standard_normal(A.n)
    f2 = f.reshape(-1, 3).copy()
    f2[:, 1:] *= s
    assert np.allclose(orc.qimpes_restrict(m["nb"], 3, w2, f2.reshape(-1)),
                       orc.qimpes_restrict(m["nb"], 3, w, f), rtol=1e-13, atol=1e-13)


def test_cpr_exact_pressure_stage_without_coupling(orc):
    """No pressure-saturation coupling and an exact pressure solve: the CPR
    apply returns the exact pressure solution (the second stage sees a zero
    pressure residual)."""
    g = synth.Grid(4, 3, 3)
    m = synth.black_oil_bsr3(g, 10)
    bv = m["bval"].reshape(-1, 3, 3).copy()
    bv[:, 0, 1:] = 0.0
    bv[:, 1:, 0] = 0.0
    A = orc.Mat(m["browptr"], m["bcol"], bv.reshape(-1), 3)
    p = synth.pressure_7pt(g, 10)
    App = sp.csr_matrix((p["val"], p["col"], p["rowptr"]), shape=(g.n, g.n)).tocsc()
    lu = spla.splu(App)
    M = orc.PC(A, "cpr", pstage=lambda rp: lu.solve(rp))
    f = np.random.default_rng(11).standard_normal(A.n)
    z = M.apply(f)
    assert np.allclose(z[0::3], lu.solve(f[0::3]), rtol=1e-12, atol=1e-12)
    # with the pressure stage dropped, CPR is block ILU(0) alone
    M0 = orc.PC(A, "cpr", pstage=lambda rp: np.zeros_like(rp))
    Mb = orc.PC(A, "bilu0")
    assert np.allclose(M0.apply(f), Mb.apply(f), rtol=1e-14, atol=1e-14)


def test_cpr_scalar_exact_stage_is_exact(orc):
    d = synth.pressure_7pt(synth.Grid(5, 4, 3), 13)
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"])).tocsc()
    lu = spla.splu(S)
    M = orc.PC(A, "cpr", pstage=lambda r: lu.solve(r))
    f = np.random.default_rng(12).standard_normal(A.n)
    assert np.allclose(M.apply(f), lu.solve(f), rtol=1e-10, atol=1e-12)


def _dense_operator(M, n):
    """The preconditioner as a dense matrix B (z = B f), column by column."""
    return np.stack([M.apply(e) for e in np.eye(n)], axis=1)


def test_cpr_forms_are_the_printed_compositions(orc):
    """Algs. 5-8 chain a pressure stage P and the block ILU(0) F through
    residual corrections, so each form's error propagator I - B A is the
    product of the stages' propagators in the printed order:
      PF: E_F E_P,  FP: E_P E_F,  FPF: E_F E_P E_F,  FFPF: E_F E_P E_F E_F.
    The stages' dense operators come from the separately pinned pieces:
    B_F from block ILU(0), B_P = Pi_p ILU0(App')^{-1} Pi_r."""
    m = synth.black_oil_bsr3(synth.Grid(3, 2, 2), 21)
    A = orc.Mat.bsr(m)
    D = _block_dense(m)
    n, nb = D.shape[0], m["nb"]
    I = np.eye(n)
    BF = _dense_operator(orc.PC(A, "bilu0"), n)
    w = orc.qimpes_weights(A)
    App = orc.Mat(m["browptr"], m["bcol"], orc.qimpes_app(A, w), 1)
    _, _, lu = orc.ilu0(App)

    def pstage(v):
        z = np.zeros(n)
        z[0::3] = orc.ilu0_solve(App, lu, orc.qimpes_restrict(nb, 3, w, v))
        return z
    BP = np.stack([pstage(e) for e in np.eye(n)], axis=1)
    EF, EP = I - BF @ D, I - BP @ D
    pred = {"pf": EF @ EP, "fp": EP @ EF, "fpf": EF @ EP @ EF, "ffpf": EF @ EP @ EF @ EF}
    for form in orc.PC.FORMS:
        E = I - _dense_operator(orc.PC(A, "cpr", form=form), n) @ D
        assert np.allclose(E, pred[form], rtol=1e-10, atol=1e-12), form


def test_cpr_forms_exact_when_block_ilu_is_exact(orc):
    """On a 1-D chain block ILU(0) is the exact block LU, so every form that
    ends with (or begins with) an F stage returns A^{-1} f."""
    m = synth.black_oil_bsr3(synth.Grid(9, 1, 1), 4)
    A = orc.Mat.bsr(m)
    D = _block_dense(m)
    f = np.random.default_rng(22).standard_normal(D.shape[0])
    x = np.linalg.solve(D, f)
    for form in orc.PC.FORMS:
        assert np.allclose(orc.PC(A, "cpr", form=form).apply(f), x, rtol=1e-10, atol=1e-11), form


# ----------------------------------------------------------------------------
# GMRES / FGMRES (Sec. 3, Alg. 1)
# ----------------------------------------------------------------------------
def test_gmres_full_space_converges_within_n(orc):
    rng = np.random.default_rng(13)
    n = 40
    D = rng.standard_normal((n, n)) + 4 * np.eye(n)
    A = orc.Mat.csr(dense_pattern_csr(D))
    b = rng.standard_normal(n)
    x, info, _ = orc.gmres(A, None, b, restart=n, rtol=1e-12, maxit=n)
    assert info["status"] == 0 and info["iters"] <= n
    assert np.allclose(x, np.linalg.solve(D, b), rtol=1e-9, atol=1e-10)


def test_gmres_poisson1d_eigenvector_one_step(orc):
    n = 50
    A = orc.Mat.csr(csr_dict(poisson1d(n)))
    v, lam = eig1d(n, 3)
    x, info, _ = orc.gmres(A, None, v, restart=30, rtol=1e-12)
    assert info["iters"] == 1 and info["status"] == 0
    assert np.allclose(x, v / lam, rtol=1e-12, atol=1e-12)


def test_gmres_q_eigenvectors_q_steps(orc):
    n = 50
    A = orc.Mat.csr(csr_dict(poisson1d(n)))
    b = sum(eig1d(n, k)[0] * c for k, c in zip((1, 4, 9, 20), (1.0, -2.0, 0.5, 3.0)))
    x, info, hist = orc.gmres(A, None, b, restart=30, rtol=1e-8, hist_len=4)
    assert info["iters"] == 4 and hist[2] > 0.1      # far from converged one step earlier
    xr = sum(eig1d(n, k)[0] * c / eig1d(n, k)[1] for k, c in zip((1, 4, 9, 20), (1.0, -2.0, 0.5, 3.0)))
    assert np.allclose(x, xr, rtol=1e-6, atol=1e-6 * np.abs(xr).max())


def test_gmres_poisson3d_dirichlet_eigenvector(orc):
    nx, ny, nz = 6, 5, 4
    A = orc.Mat.csr(csr_dict(poisson3d_dirichlet(nx, ny, nz)))
    vx, lx = eig1d(nx, 2)
    vy, ly = eig1d(ny, 1)
    vz, lz = eig1d(nz, 3)
    v = np.einsum("k,j,i->kji", vz, vy, vx).reshape(-1)
    for solver in ("gmres", "bicgstab"):
        if solver == "gmres":
            x, info, _ = orc.gmres(A, None, v, rtol=1e-12)
        else:
            x, info, _ = orc.bicgstab(A, None, v, rtol=1e-12)
        assert info["iters"] == 1, solver
        assert np.allclose(x, v / (lx + ly + lz), rtol=1e-12, atol=1e-13)


def test_cgs2_arnoldi_relation(orc):
    """A M^{-1} V_m = V_{m+1} Hbar and V^T V = I for the CGS2 step."""
    d = synth.pressure_7pt(synth.Grid(6, 6, 5), 14)
    A = orc.Mat.csr(d)
    M = orc.PC(A, "ilu0")
    n, m = d["n"], 12
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    r = np.random.default_rng(15).standard_normal(n)
    V[0] = r / np.linalg.norm(r)
    for i in range(m):
        w = orc.spmv(A, M.apply(V[i]))
        w, h = orc.orthogonalise(V[:i + 1], w, i)
        H[:i + 2, i] = h
        V[i + 1] = w / h[i + 1]
    AMV = np.stack([orc.spmv(A, M.apply(V[i])) for i in range(m)])
    assert np.abs(AMV.T - V.T @ H).max() <= 1e-12 * np.abs(AMV).max()
    assert np.abs(V @ V.T - np.eye(m + 1)).max() <= 1e-12
    # the MGS variant builds the same Hessenberg matrix (up to rounding)
    w0 = orc.spmv(A, M.apply(V[m - 1]))
    _, h_c = orc.orthogonalise(V[:m], w0, m - 1)
    _, h_m = orc.orthogonalise(V[:m], w0, m - 1, mgs=True)
    assert np.allclose(h_c, h_m, rtol=1e-10, atol=1e-12)


def test_gmres_ilu0_matches_direct_solution(orc):
    d = synth.pressure_7pt(synth.Grid(8, 8, 8), 16)
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]))
    xt = synth.x_true(d["n"], 16)
    b = S @ xt
    M = orc.PC(A, "ilu0")
    for kw in (dict(), dict(mgs=True), dict(flexible=True)):
        x, info, _ = orc.gmres(A, M, b, restart=30, rtol=1e-12, **kw)
        assert info["status"] == 0
        assert np.linalg.norm(b - S @ x) <= 1e-12 * np.linalg.norm(b) * 1.0001
        assert np.linalg.norm(x - spla.spsolve(S.tocsc(), b)) <= 1e-6 * np.linalg.norm(xt)
    x, info, _ = orc.gmres(A, M, b, restart=30, rtol=1e-12, side="left")
    assert info["status"] == 0
    assert np.linalg.norm(x - spla.spsolve(S.tocsc(), b)) <= 1e-6 * np.linalg.norm(xt)


def test_gmres_mgs_and_cgs2_iteration_counts_agree(orc):
    d = synth.pressure_7pt(synth.Grid(16, 16, 16), 17)
    A = orc.Mat.csr(d)
    b = orc.spmv(A, synth.x_true(d["n"], 17))
    M = orc.PC(A, "ilu0")
    _, i1, _ = orc.gmres(A, M, b)
    _, i2, _ = orc.gmres(A, M, b, mgs=True)
    assert abs(i1["iters"] - i2["iters"]) <= 2


def test_gmres_exact_preconditioner_one_step(orc):
    d = synth.pressure_7pt(synth.Grid(5, 5, 4), 18)
    A = orc.Mat.csr(d)
    lu = spla.splu(sp.csr_matrix((d["val"], d["col"], d["rowptr"])).tocsc())
    M = orc.PC(A, "callback", fn=lambda r: lu.solve(r))
    b = np.random.default_rng(19).standard_normal(d["n"])
    for flexible in (False, True):
        x, info, _ = orc.gmres(A, M, b, rtol=1e-10, flexible=flexible)
        assert info["iters"] == 1
    x, info, _ = orc.gmres(A, M, b, rtol=1e-10, side="left")
    assert info["iters"] == 1
    x, info, _ = orc.bicgstab(A, M, b, rtol=1e-10)
    assert info["iters"] == 1


def test_fgmres_equals_gmres_for_fixed_preconditioner(orc):
    d = synth.pressure_7pt(synth.Grid(10, 9, 8), 20)
    A = orc.Mat.csr(d)
    b = orc.spmv(A, synth.x_true(d["n"], 20))
    M = orc.PC(A, "ilu0")
    for maxit in (7, 30, 47):
        x1, i1, h1 = orc.gmres(A, M, b, restart=20, rtol=1e-14, maxit=maxit, hist_len=maxit)
        x2, i2, h2 = orc.fgmres(A, M, b, restart=20, rtol=1e-14, maxit=maxit, hist_len=maxit)
        assert i1["iters"] == i2["iters"] == maxit
        assert np.allclose(x1, x2, rtol=1e-12, atol=1e-12 * np.abs(x1).max())
        assert np.allclose(h1, h2, rtol=1e-10)


def test_gmres_edge_cases(orc):
    d = synth.pressure_7pt(synth.Grid(4, 4, 4), 21)
    A = orc.Mat.csr(d)
    x, info, _ = orc.gmres(A, None, np.zeros(d["n"]), x0=np.ones(d["n"]))
    assert info["status"] == 0 and info["iters"] == 0 and (x == 0).all()
    xt = synth.x_true(d["n"], 21)
    b = orc.spmv(A, xt)
    x, info, _ = orc.gmres(A, None, b, maxit=5)
    assert info["status"] == orc.NOT_CONVERGED and info["iters"] == 5
    x, info, _ = orc.gmres(A, None, b, x0=xt)
    assert info["status"] == 0 and info["iters"] == 0


# ----------------------------------------------------------------------------
# BiCGSTAB
# ----------------------------------------------------------------------------
def test_bicgstab_matches_direct_and_breakdown(orc):
    d = synth.pressure_7pt(synth.Grid(8, 7, 6), 22, kz_scale=0.1)
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]))
    b = S @ synth.x_true(d["n"], 22)
    for M in (None, orc.PC(A, "ilu0")):
        x, info, _ = orc.bicgstab(A, M, b, rtol=1e-12)
        assert info["status"] == 0
        assert np.linalg.norm(b - S @ x) <= 1e-12 * np.linalg.norm(b) * 1.0001
        assert np.allclose(x, spla.spsolve(S.tocsc(), b), rtol=1e-8, atol=1e-8)
    # (rhat, A p) = 0 on the first step: A = [[0,1],[1,0]], b = e1
    B = orc.Mat.csr(csr_dict(np.array([[0.0, 1.0], [1.0, 0.0]])))
    _, info, _ = orc.bicgstab(B, None, np.array([1.0, 0.0]))
    assert info["status"] == orc.BREAKDOWN


def test_bicgstab_single_eigvec_and_spd_count(orc):
    n = 60
    A = orc.Mat.csr(csr_dict(poisson1d(n)))
    v, lam = eig1d(n, 5)
    x, info, _ = orc.bicgstab(A, None, v, rtol=1e-12)
    assert info["iters"] == 1 and np.allclose(x, v / lam, rtol=1e-12, atol=1e-13)


# ----------------------------------------------------------------------------
# CG (Alg. 2)
# ----------------------------------------------------------------------------
def test_cg_eigenvectors_and_finite_termination(orc):
    """Unpreconditioned CG on the 1-D Dirichlet Poisson matrix: one step for
    an eigenvector (x = v / lambda), q steps for q eigenvectors, at most n
    steps for any right-hand side (finite termination on SPD systems)."""
    n = 50
    A = orc.Mat.csr(csr_dict(poisson1d(n)))
    v, lam = eig1d(n, 7)
    x, info, _ = orc.cg(A, None, v, rtol=1e-12)
    assert info["iters"] == 1 and info["status"] == 0
    assert np.allclose(x, v / lam, rtol=1e-12, atol=1e-13)
    ks, cs = (2, 5, 11, 30), (1.0, -0.5, 2.0, 0.25)
    b = sum(eig1d(n, k)[0] * c for k, c in zip(ks, cs))
    x, info, hist = orc.cg(A, None, b, rtol=1e-8, hist_len=4)
    assert info["iters"] == 4 and hist[2] > 1e-3
    xr = sum(eig1d(n, k)[0] * c / eig1d(n, k)[1] for k, c in zip(ks, cs))
    assert np.allclose(x, xr, rtol=1e-6, atol=1e-6 * np.abs(xr).max())
    b = np.random.default_rng(31).standard_normal(n)
    x, info, _ = orc.cg(A, None, b, rtol=1e-10, maxit=10 * n)
    assert info["status"] == 0 and info["iters"] <= n
    assert np.allclose(poisson1d(n) @ x, b, rtol=1e-9, atol=1e-9)


def test_cg_exact_preconditioner_and_breakdown(orc):
    """With M = A (dense solve as the preconditioner) CG converges in one
    step; on an indefinite matrix (p, A p) = 0 is reported as a breakdown."""
    d = synth.pressure_7pt(synth.Grid(6, 5, 4), 32)
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"])).tocsc()
    lu = spla.splu(S)
    b = orc.spmv(A, synth.x_true(d["n"], 32))
    x, info, _ = orc.cg(A, orc.PC(A, "callback", fn=lambda r: lu.solve(r)), b, rtol=1e-12)
    assert info["iters"] == 1 and info["status"] == 0
    assert np.allclose(x, lu.solve(b), rtol=1e-10, atol=1e-12)
    x, info, _ = orc.cg(A, orc.PC(A, "ilu0"), b, rtol=1e-10)
    assert info["status"] == 0 and info["true_rel_res"] <= 1e-10
    B = orc.Mat.csr(csr_dict(np.array([[0.0, 1.0], [1.0, 0.0]])))
    _, info, _ = orc.cg(B, None, np.array([1.0, 0.0]))
    assert info["status"] == orc.BREAKDOWN


def test_mixed_precision_preconditioners_converge(orc):
    d = synth.pressure_7pt(synth.Grid(12, 12, 8), 23, kz_scale=0.1)
    A = orc.Mat.csr(d)
    b = orc.spmv(A, synth.x_true(d["n"], 23))
    x64, i64, _ = orc.gmres(A, orc.PC(A, "ilu0"), b)
    x32, i32, _ = orc.gmres(A, orc.PC(A, "ilu0", mixed=True), b)
    assert i32["status"] == 0 and i32["true_rel_res"] <= 1e-8
    assert abs(i32["iters"] - i64["iters"]) <= 3


# ----------------------------------------------------------------------------
# ILU(k) patterns and restricted additive Schwarz (Sec. 4.1)
# ----------------------------------------------------------------------------
def _fill_path_pattern(P, p):
    """Brute force of the fill-path theorem (Rose-Tarjan; Hysom-Pothen for the
    sum rule of levels): (i, j) has level <= p iff the directed graph of P
    holds a path i -> j of at most p + 1 edges whose inner vertices are all
    numbered below min(i, j)."""
    n = P.shape[0]
    keep = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for j in range(n):
            m = min(i, j)
            found = bool(P[i, j]) or i == j
            seen, frontier, d = {i}, [i], 0
            while frontier and not found and d < p + 1:
                d += 1
                nxt = []
                for u in frontier:
                    for v in np.nonzero(P[u])[0]:
                        if v == j:
                            found = True
                        elif v < m and v not in seen:
                            seen.add(v)
                            nxt.append(v)
                frontier = nxt
            keep[i, j] = found
    return keep


def test_iluk_pattern_is_the_fill_path_pattern(orc):
    rng = np.random.default_rng(40)
    for trial in range(4):
        n = 24
        P = (rng.random((n, n)) < 0.09) | np.eye(n, dtype=bool)
        d = csr_dict(sp.csr_matrix(P.astype(float)))
        for p in (0, 1, 2, 3):
            ptr, col = orc.iluk_pattern(n, d["rowptr"], d["col"], p)
            got = np.zeros((n, n), dtype=bool)
            for i in range(n):
                cols = col[ptr[i]:ptr[i + 1]]
                assert (np.diff(cols) > 0).all()                     # sorted, no duplicates
                got[i, cols] = True
            assert np.array_equal(got, _fill_path_pattern(P, p)), (trial, p)


def _ilu_on_pattern(orc, d, level):
    """ILU(level) of d through the one-subdomain Schwarz object (no overlap):
    the stacked matrix is then the matrix itself."""
    R = orc.Ras(orc.Mat.csr(d), 1, overlap=0, level=level)
    assert R.status == 0
    gidx, ptr, col, lu = R.structure()
    assert np.array_equal(gidx, np.arange(d["n"]))
    return ptr, col, lu


def test_iluk_numeric_invariant_7pt(orc):
    g = synth.Grid(5, 4, 3)
    d = synth.pressure_7pt(g, 41)
    A = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(g.n, g.n)).toarray()
    prev = A != 0
    for level in (1, 2):
        ptr, col, lu = _ilu_on_pattern(orc, d, level)
        e = dict(n=g.n, rowptr=ptr, col=col)
        L, U = lu_dense_from_ilu(e, lu)
        P = np.zeros_like(prev)
        for i in range(g.n):
            P[i, col[ptr[i]:ptr[i + 1]]] = True
        assert (P & prev == prev).all() and P.sum() > prev.sum()      # the pattern only grows
        LU = L @ U
        assert np.allclose(LU[P], A[P], rtol=1e-13, atol=1e-13)       # (LU)_ij = a_ij on the ILU(k) pattern
        assert (np.tril(L, -1)[~P] == 0).all() and (U[~P] == 0).all()
        prev = P
    # a 1-D chain has no fill at any level: ILU(k) = ILU(0) = the exact LU
    d1 = csr_dict(poisson1d(30))
    ptr, col, lu = _ilu_on_pattern(orc, d1, 3)
    assert np.array_equal(ptr, d1["rowptr"]) and np.array_equal(col, d1["col"])
    L, U = lu_dense_from_ilu(d1, lu)
    assert np.allclose(L @ U, poisson1d(30).toarray(), atol=1e-14)


def test_ras_one_subdomain_without_overlap_is_ilu0(orc):
    d = synth.pressure_7pt(synth.Grid(6, 5, 4), 42)
    A = orc.Mat.csr(d)
    r = synth.x_true(d["n"], 43)
    _, _, lu = orc.ilu0(A)
    z = orc.Ras(A, 1, overlap=0, level=0).apply(r)
    assert np.array_equal(z, orc.ilu0_solve(A, lu, r))


def test_ras_one_row_per_subdomain_is_jacobi(orc):
    d = synth.pressure_7pt(synth.Grid(5, 4, 3), 44)
    n = d["n"]
    A = orc.Mat.csr(d)
    diag = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(n, n)).diagonal()
    r = synth.x_true(n, 45)
    z = orc.Ras(A, n, part=np.arange(n, dtype=np.int32), overlap=0).apply(r)
    assert np.array_equal(z, r / diag)


def _extended_sets(S, part, nsub, overlap):
    G = (S != 0).toarray()
    sets = []
    for s in range(nsub):
        m = part == s
        for _ in range(overlap):
            m = m | G[m].any(axis=0)
        sets.append(np.nonzero(m)[0])
    return sets


def test_ras_on_a_chain_is_the_restricted_block_solve(orc):
    # on a tridiagonal matrix every local ILU(0) is the exact LU of the local
    # matrix, so RAS is: solve densely on each extended set, keep owned rows
    rng = np.random.default_rng(46)
    n = 50
    D = np.diag(3 + rng.random(n)) + np.diag(-rng.random(n - 1), 1) + np.diag(-rng.random(n - 1), -1)
    S = sp.csr_matrix(D)
    A = orc.Mat.csr(csr_dict(D))
    r = rng.standard_normal(n)
    parts = [orc.contiguous_partition(n, 4), rng.integers(0, 5, n).astype(np.int32)]
    for part in parts:
        nsub = int(part.max()) + 1
        for overlap in (0, 1, 3):
            z = orc.Ras(A, nsub, part=part, overlap=overlap).apply(r)
            want = np.empty(n)
            for s, e in enumerate(_extended_sets(S, part, nsub, overlap)):
                if e.size == 0:
                    continue
                ze = np.linalg.solve(D[np.ix_(e, e)], r[e])
                own = part[e] == s
                want[e[own]] = ze[own]
            assert np.allclose(z, want, rtol=1e-13, atol=1e-13), (nsub, overlap)
    # overlap reaching every row: each subdomain solves the whole system
    z = orc.Ras(A, 3, overlap=n, level=0).apply(r)
    assert np.allclose(z, np.linalg.solve(D, r), rtol=1e-12, atol=1e-12)


def test_ras_structure_and_invalid_inputs(orc):
    d = synth.pressure_7pt(synth.Grid(6, 6, 4), 47)
    n = d["n"]
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(n, n))
    part = orc.contiguous_partition(n, 3)
    R = orc.Ras(A, 3, part=part, overlap=2, level=1)
    gidx, ptr, col, lu = R.structure()
    sets = _extended_sets(S, part, 3, 2)
    assert np.array_equal(gidx, np.concatenate(sets))
    base = np.cumsum([0] + [len(e) for e in sets])
    for s in range(3):                                   # columns stay inside their block
        rows = slice(base[s], base[s + 1])
        c = col[ptr[base[s]]:ptr[base[s + 1]]]
        assert c.min() >= base[s] and c.max() < base[s + 1]
        assert rows.stop - rows.start == len(sets[s])
    assert orc.Ras(A, 3, part=np.full(n, 3, np.int32)).status == orc.INVALID
    assert orc.Ras(A, 0).status == orc.INVALID
    assert orc.Ras(A, 2, overlap=-1).status == orc.INVALID


def test_ras_gmres_converges_and_overlap_helps(orc):
    d = synth.pressure_7pt(synth.Grid(12, 12, 12), 48)
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]))
    b = S @ synth.x_true(d["n"], 48)
    its = {}
    for overlap in (0, 2):
        for level in (0, 1):
            M = orc.PC(A, "ras", ras=dict(nsub=8, overlap=overlap, level=level))
            x, info, _ = orc.gmres(A, M, b, restart=30, rtol=1e-10)
            assert info["status"] == 0
            assert np.linalg.norm(b - S @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001
            its[overlap, level] = info["iters"]
    assert its[2, 0] < its[0, 0] and its[2, 1] < its[0, 1]


# ----------------------------------------------------------------------------
# Algebraic multigrid (Sec. 4.2, Algs. 3-4, Eq. 4)
# ----------------------------------------------------------------------------
def _csr_dense(t, m=None):
    ptr, col, val = t
    n = ptr.size - 1
    return sp.csr_matrix((val, col, ptr), shape=(n, m if m is not None else n)).toarray()


def test_amg_poisson1d_is_geometric_multigrid(orc):
    # 1-D Poisson, 2^4 - 1 points: Ruge-Stueben picks every other point,
    # direct interpolation is linear interpolation and the Galerkin matrix is
    # (1/2) tridiag(-1, 2, -1): each level is the previous one halved
    M = orc.Amg(orc.Mat.csr(csr_dict(poisson1d(15))), max_coarse=1, coarsen="rs")
    assert M.status == 0
    lv = M.levels()
    assert [a[0].size - 1 for a, _ in lv] == [15, 7, 3, 1]
    for l, (a, p) in enumerate(lv[:-1]):
        n = a[0].size - 1
        nc = (n - 1) // 2
        Pd = _csr_dense(p, nc)
        want = np.zeros((n, nc))
        for k in range(nc):                       # coarse point k is fine point 2k + 1
            want[2 * k + 1, k] = 1.0
            want[2 * k, k] = want[2 * k + 2, k] = 0.5
        assert np.array_equal(Pd, want)
        Ac = _csr_dense(lv[l + 1][0])
        assert np.allclose(Ac, 0.5 ** (l + 1) * poisson1d(nc).toarray(), rtol=0, atol=1e-15)


def test_amg_anisotropy_gives_semicoarsening(orc):
    # 2-D Laplacian with weak y couplings (eps = 0.1 < theta = 0.5): only x
    # couplings are strong, so every x-line is coarsened alone, every other
    # point (Ruge-Stueben's textbook semicoarsening)
    nx, ny, eps = 9, 6, 0.1
    Ax = poisson1d(nx)
    Ay = poisson1d(ny)
    A = (sp.kron(sp.eye(ny), Ax) + eps * sp.kron(Ay, sp.eye(nx))).tocsr()
    M = orc.Amg(orc.Mat.csr(csr_dict(A)), max_levels=2, max_coarse=1, coarsen="rs")
    a, p = M.levels()[0]
    Pd = _csr_dense(p, 4 * ny)
    C = [i for i in range(nx * ny) if (Pd[i] != 0).sum() == 1 and Pd[i].max() == 1.0]   # injected points
    assert C == [y * nx + x for y in range(ny) for x in (1, 3, 5, 7)]


def test_splitmix64_published_outputs(orc):
    # SplitMix64 from state 0 (Steele, Lea and Flood 2014): its first outputs
    assert [orc.splitmix64(k) for k in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def _chain_strength(n):
    # 1-D Poisson with theta = 0.5: both neighbours of a point are strong
    ptr, col = [0], []
    for i in range(n):
        col += [j for j in (i - 1, i + 1) if 0 <= j < n]
        ptr.append(len(col))
    return np.array(ptr, np.int32), np.array(col, np.int32)


def test_pmis_hand_worked_chains(orc):
    # 7 points in a chain; lambda_i = |S_i^T| + w_i = 2 + w_i inside, 1 + w_i
    # at the ends.  (a) w = .1 .5 .2 .9 .3 .4 .8: lambda = 1.1 2.5 2.2 2.9
    # 2.3 2.4 1.8; the local maxima 1, 3, 5 become C in the first round and
    # their neighbours F.  (b) w rising .1 .2 ... .7: lambda = 1.1 2.2 2.3
    # 2.4 2.5 2.6 1.7; round 1 takes 5 (4 and 6 become F), round 2 takes 3
    # among the undecided 0..3 (2 becomes F), round 3 takes 1 (0 becomes F)
    sptr, scol = _chain_strength(7)
    st, rounds = orc.pmis(7, sptr, scol, [.1, .5, .2, .9, .3, .4, .8])
    assert st.tolist() == [2, 1, 2, 1, 2, 1, 2] and rounds == 1
    st, rounds = orc.pmis(7, sptr, scol, [.1, .2, .3, .4, .5, .6, .7])
    assert st.tolist() == [2, 1, 2, 1, 2, 1, 2] and rounds == 3
    # a point that influences nothing is F from the start, even with the
    # largest weight; a point with no neighbour left undecided becomes C
    sptr = np.array([0, 1, 2, 2], np.int32)
    scol = np.array([1, 0], np.int32)          # 0 and 1 depend on each other; 2 is isolated
    st, _ = orc.pmis(3, sptr, scol, [.3, .2, .99])
    assert st.tolist() == [1, 2, 2]


@pytest.mark.parametrize("shape,kz,seed", [((9, 8, 7), 1.0, 70), ((12, 10, 6), 0.1, 71)])
def test_pmis_invariants(orc, shape, kz, seed):
    """On 7-point systems with the SplitMix64 weights: every point is decided;
    every F point either influences no point or depends strongly on a C
    point; for two strongly coupled C points the one of smaller measure does
    not depend strongly on the other (it stayed undecided after the other
    became C, so it cannot depend on it)."""
    g = synth.Grid(*shape)
    d = synth.pressure_7pt(g, seed, kz_scale=kz)
    A = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(g.n, g.n))
    n, theta = g.n, 0.5
    S = []
    for i in range(n):
        row = A.getrow(i)
        off = [(j, v) for j, v in zip(row.indices, row.data) if j != i]
        mx = max([-v for _, v in off] + [0.0])
        S.append(sorted(j for j, v in off if mx > 0 and -v >= theta * mx))
    sptr = np.cumsum([0] + [len(x) for x in S]).astype(np.int32)
    scol = np.array([j for x in S for j in x], np.int32)
    w = np.array([(orc.splitmix64((0 << 32) | i) >> 11) * 2.0 ** -53 for i in range(n)])
    st, rounds = orc.pmis(n, sptr, scol, w)
    assert set(st.tolist()) <= {1, 2} and rounds >= 2
    infl = np.zeros(n, int)
    for x in S:
        for j in x:
            infl[j] += 1
    lam = infl + w
    for i in range(n):
        if st[i] == 2:
            assert infl[i] == 0 or any(st[j] == 1 for j in S[i]), i
        else:
            for j in S[i]:
                if st[j] == 1:
                    assert lam[j] > lam[i] or i not in S[j], (i, j)
    # the C points of the oracle's first AMG level are these
    M = orc.Amg(orc.Mat.csr(d), max_levels=2, max_coarse=1)
    assert np.array_equal(M.cidx(0) >= 0, st == 1)


def test_amg_pmis_galerkin_and_convergence(orc):
    # with PMIS coarsening the coarse matrices are still P^T A P (Eq. 4) and
    # PCG with one V-cycle converges in a bounded number of iterations
    g = synth.Grid(16, 14, 12)
    d = synth.pressure_7pt(g, 63)
    M = orc.Amg(orc.Mat.csr(d), max_coarse=16)
    assert M.status == 0
    lv = M.levels()
    assert len(lv) >= 3
    for l, (a, p) in enumerate(lv[:-1]):
        Ad = _csr_dense(a)
        nc = lv[l + 1][0][0].size - 1
        Pd = _csr_dense(p, nc)
        assert np.allclose(_csr_dense(lv[l + 1][0]), Pd.T @ Ad @ Pd, rtol=0, atol=1e-12 * np.abs(Ad).max())
    Ao = orc.Mat.csr(d)
    b = orc.spmv(Ao, synth.x_true(g.n, 63))
    x, info, _ = orc.cg(Ao, orc.PC(Ao, "amg", amg=dict(max_coarse=16)), b, rtol=1e-8)
    assert info["status"] == 0 and info["iters"] <= 30, info


def test_amg_galerkin_and_constant_interpolation(orc):
    # A_{l+1} = P^T A_l P on every level (Eq. 4); on a zero-row-sum matrix
    # direct interpolation reproduces constants: every row of P sums to 1
    g = synth.Grid(7, 6, 5)
    d = synth.pressure_7pt(g, 60, accum=0.0)
    n = g.n
    d["val"] = d["val"].copy()
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(n, n))
    assert np.abs(S.sum(axis=1)).max() < 1e-12
    # pin the singular matrix's coarsest level away from it: add 1e-3 to one diagonal entry
    dd = np.nonzero(d["col"] == np.repeat(np.arange(n), np.diff(d["rowptr"])))[0]
    d["val"][dd[0]] += 1e-3
    M = orc.Amg(orc.Mat.csr(d), max_coarse=8, coarsen="rs")
    assert M.status == 0
    lv = M.levels()
    assert len(lv) >= 3
    for l, (a, p) in enumerate(lv[:-1]):
        Ad = _csr_dense(a)
        nc = lv[l + 1][0][0].size - 1
        Pd = _csr_dense(p, nc)
        assert np.allclose(_csr_dense(lv[l + 1][0]), Pd.T @ Ad @ Pd, rtol=0, atol=1e-12 * np.abs(Ad).max())
        # rows of A_l that sum to zero (all but those the shift reaches) interpolate constants exactly
        zero = np.abs(Ad.sum(axis=1)) <= 1e-12 * np.abs(Ad).max()
        rows = zero & (Pd != 0).any(axis=1)
        assert rows.sum() > (0.5 * Pd.shape[0] if l == 0 else 0)
        assert np.allclose(Pd.sum(axis=1)[rows], 1.0, rtol=0, atol=1e-12)


def test_amg_vcycle_is_symmetric_positive_definite(orc):
    # pre- and post-smoothing by the same l1-Jacobi sweeps and R = P^T make
    # the V-cycle a symmetric positive definite operator for SPD A
    g = synth.Grid(6, 5, 4)
    d = synth.pressure_7pt(g, 61)
    M = orc.Amg(orc.Mat.csr(d), max_coarse=10)
    assert len(M.levels()) >= 3
    B = np.column_stack([M.apply(e) for e in np.eye(g.n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_amg_pcg_iterations_do_not_grow_with_the_grid(orc):
    its = []
    for m in (10, 20):
        A = poisson3d_dirichlet(m, m, m)
        d = csr_dict(A)
        Ao = orc.Mat.csr(d)
        b = A @ np.random.default_rng(62).standard_normal(m ** 3)
        Mo = orc.PC(Ao, "amg", amg=dict(max_coarse=32))
        x, info, _ = orc.cg(Ao, Mo, b, rtol=1e-8)
        assert info["status"] == 0
        assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001
        its.append(info["iters"])
    assert its[1] <= its[0] + 3 and its[1] <= 20, its


def _hgs_by_library(A, b, x, chunk, backward):
    """A hybrid Gauss-Seidel sweep as one block-diagonal triangular solve:
    x + (D + T_C)^{-1} (b - A x), T_C the strictly lower (backward: upper)
    part of A kept only inside a chunk of consecutive rows, solved by scipy's
    sparse triangular solver (the Gauss-Seidel splitting, chunk by chunk)."""
    C = A.tocoo()
    same = (C.row // chunk) == (C.col // chunk)
    tri = (C.col > C.row) if backward else (C.col < C.row)
    keep = (C.row == C.col) | (same & tri)
    T = sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)
    return x + spla.spsolve_triangular(T, b - A @ x, lower=not backward)


@pytest.mark.parametrize("chunk", [1, 7, 32, 1000])
@pytest.mark.parametrize("backward", [False, True])
def test_hybrid_gauss_seidel_sweep_is_a_chunked_triangular_solve(orc, chunk, backward):
    """Fig. 34's relaxation (Gauss-Seidel inside a process, Jacobi between
    processes) with 32-row chunks as the processes: checked against the
    splitting solved by a library triangular solver, on a nonsymmetric
    matrix with a ragged last chunk; chunk 1 is Jacobi, a chunk larger than
    the matrix plain Gauss-Seidel."""
    rng = np.random.default_rng(71)
    n = 100
    R = sp.random(n, n, density=0.08, random_state=72, format="csr")
    A = (R - R.T * 0.5 + sp.diags(np.abs(R).sum(axis=1).A1 + 2.0 + rng.random(n))).tocsr()
    A.sort_indices()
    Ao = orc.Mat.csr(csr_dict(A))
    b = rng.standard_normal(n)
    x = rng.standard_normal(n)
    st, got = orc.hgs_sweep(Ao, b, x, chunk=chunk, backward=backward)
    assert st == orc.OK
    ref = _hgs_by_library(A, b, x, chunk, backward)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    if chunk == 1:
        d = A.diagonal()
        assert np.allclose(got, x + (b - A @ x) / d, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_amg_hybrid_gauss_seidel_vcycle_is_spd_and_beats_l1_jacobi(orc):
    """Forward sweeps before the coarse correction and backward sweeps after
    it are adjoint for symmetric A, so the V-cycle stays symmetric positive
    definite; as the stronger smoother it needs no more CG iterations than
    l1-Jacobi, and it still does not grow with the grid."""
    g = synth.Grid(6, 5, 4)
    d = synth.pressure_7pt(g, 61)
    M = orc.Amg(orc.Mat.csr(d), max_coarse=10, smoother=1)
    assert M.status == orc.OK and len(M.levels()) >= 3
    B = np.column_stack([M.apply(e) for e in np.eye(g.n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    its = {}
    for m in (10, 20):
        A = poisson3d_dirichlet(m, m, m)
        Ao = orc.Mat.csr(csr_dict(A))
        b = A @ np.random.default_rng(62).standard_normal(m ** 3)
        for sm in (0, 1):
            x, info, _ = orc.cg(Ao, orc.PC(Ao, "amg", amg=dict(max_coarse=32, smoother=sm)), b, rtol=1e-8)
            assert info["status"] == 0
            assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001
            its[m, sm] = info["iters"]
    assert its[10, 1] <= its[10, 0] and its[20, 1] <= its[20, 0], its
    assert its[20, 1] <= its[10, 1] + 3, its


def test_amg_hybrid_gauss_seidel_needs_a_diagonal(orc):
    A = poisson1d(10).tolil()
    A[3, 3] = 0.0
    A = A.tocsr()
    A.eliminate_zeros()
    Ao = orc.Mat.csr(csr_dict(A))
    assert orc.Amg(Ao, smoother=1).status == orc.ZERO_PIVOT
    assert orc.Amg(Ao, smoother=0).status == orc.OK
    assert orc.Amg(orc.Mat.csr(csr_dict(poisson1d(10))), smoother=2).status == orc.INVALID


def test_amg_invalid_inputs(orc):
    A = orc.Mat.csr(csr_dict(poisson1d(10)))
    assert orc.Amg(A, max_levels=0).status == orc.INVALID
    assert orc.Amg(A, nu=0).status == orc.INVALID
    assert orc.Amg(A, theta=-1.0).status == orc.INVALID


def _rs_first_pass_by_definition(A, theta):
    """The Ruge-Stueben first pass from its definition, recomputing the
    measure of every undecided point at every step instead of updating it:
    lambda_i = |S_i^T n U| + 2 |S_i^T n F| (S_i = points strongly influencing
    i); pick the largest lambda, lowest index on ties; the new C point's
    undecided dependents become F.  Points with no strong connection in
    either direction are F from the start."""
    D = A.toarray()
    n = D.shape[0]
    S = np.zeros((n, n), dtype=bool)                  # S[i, j]: j strongly influences i
    for i in range(n):
        off = -np.delete(D[i], i)
        mx = off.max() if n > 1 else 0.0
        if mx > 0:
            for j in range(n):
                if j != i and -D[i, j] >= theta * mx:
                    S[i, j] = True
    U, Cp, Fp = 0, 1, 2
    st = np.zeros(n, int)
    for i in range(n):
        if not S[i].any() and not S[:, i].any():
            st[i] = Fp
    while (st == U).any():
        lam = np.array([(S[:, i] & (st == U)).sum() + 2 * (S[:, i] & (st == Fp)).sum() for i in range(n)])
        lam[st != U] = -1
        i = int(np.argmax(lam))                       # first maximum = lowest index
        st[i] = Cp
        for j in np.nonzero(S[:, i] & (st == U))[0]:
            st[j] = Fp
    return st == Cp


def test_amg_coarsening_follows_the_first_pass_definition(orc):
    rng = np.random.default_rng(63)
    for trial in range(12):
        n = 40
        W = rng.random((n, n)) < 0.1                        # nonsymmetric strength: the measure's
        D = np.where(W, -rng.random((n, n)), 0.0)           # decrements for the new C point matter
        np.fill_diagonal(D, 0.0)
        np.fill_diagonal(D, -D.sum(axis=1) + 0.1)
        A = sp.csr_matrix(D)
        M = orc.Amg(orc.Mat.csr(csr_dict(A)), max_levels=2, max_coarse=1, coarsen="rs")
        assert M.status == 0
        assert np.array_equal(M.cidx(0) >= 0, _rs_first_pass_by_definition(A, 0.5)), trial
    # the isotropic 5-point Laplacian coarsens red-black
    nx, ny = 8, 7
    A = (sp.kron(sp.eye(ny), poisson1d(nx)) + sp.kron(poisson1d(ny), sp.eye(nx))).tocsr()
    c = orc.Amg(orc.Mat.csr(csr_dict(A)), max_levels=2, max_coarse=1, coarsen="rs").cidx(0) >= 0
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    assert np.array_equal(c, ((x + y) % 2 == 0).reshape(-1))


def test_cpr_with_amg_pressure_stage_is_the_composition(orc):
    # CPR-PF on a scalar matrix with an AMG pressure stage: z1 = AMG(f),
    # t = f - A z1, z = z1 + ILU(0)^{-1} t, from the separately pinned pieces
    d = synth.pressure_7pt(synth.Grid(9, 8, 7), 64)
    A = orc.Mat.csr(d)
    f = synth.x_true(d["n"], 64)
    M = orc.PC(A, "cpr", amg=dict(max_coarse=20))
    z1 = orc.Amg(A, max_coarse=20).apply(f)
    _, _, lu = orc.ilu0(A)
    want = z1 + orc.ilu0_solve(A, lu, f - orc.spmv(A, z1))
    assert np.allclose(M.apply(f), want, rtol=1e-14, atol=1e-14)


# ----------------------------------------------------------------------------
# LGMRES (the aug_k of Sec. 3's solver settings)
# ----------------------------------------------------------------------------
def _nonsymmetric(n, seed):
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((n, n)) / np.sqrt(n) + 2.5 * np.eye(n)
    return D, csr_dict(D)


def test_lgmres_without_augmentation_is_fgmres(orc):
    D, d = _nonsymmetric(60, 90)
    A = orc.Mat.csr(d)
    b = np.random.default_rng(91).standard_normal(60)
    M = orc.PC(A, "ilu0")
    x1, i1 = orc.lgmres(A, M, b, restart=7, aug_k=0, rtol=1e-10)
    x2, i2, _ = orc.gmres(A, M, b, restart=7, rtol=1e-10, flexible=True)
    assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)


def test_lgmres_second_cycle_minimises_over_the_augmented_space(orc):
    # cycle 2 minimises ||b - A x|| over x1 + K_m(A, r1) + span{x1 - x0}: the
    # dense least-squares solution over that space, computed from scratch
    n, m = 40, 4
    D, d = _nonsymmetric(n, 92)
    A = orc.Mat.csr(d)
    b = np.random.default_rng(93).standard_normal(n)
    x0 = np.random.default_rng(95).standard_normal(n)
    x1, i1 = orc.lgmres(A, None, b, x0=x0, restart=m, aug_k=1, rtol=1e-15, maxit=m)
    assert i1["iters"] == m
    x2, i2 = orc.lgmres(A, None, b, x0=x0, restart=m, aug_k=1, rtol=1e-15, maxit=2 * m + 1)
    assert i2["iters"] == 2 * m + 1
    r1 = b - D @ x1
    K = [r1]
    for _ in range(m - 1):
        K.append(D @ K[-1])
    B = np.column_stack(K + [x1 - x0])
    y = np.linalg.lstsq(D @ B, r1, rcond=None)[0]
    want = x1 + B @ y
    assert np.linalg.norm(x2 - want) <= 1e-9 * np.linalg.norm(want)
    # and it is at least as good as plain GMRES over the Krylov part alone
    y0 = np.linalg.lstsq(D @ B[:, :m], r1, rcond=None)[0]
    assert np.linalg.norm(b - D @ x2) <= np.linalg.norm(r1 - D @ B[:, :m] @ y0) * (1 + 1e-12)


def test_lgmres_converges_with_ilu0(orc):
    d = synth.pressure_7pt(synth.Grid(12, 10, 8), 94, kz_scale=0.1)
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]))
    b = S @ synth.x_true(d["n"], 94)
    x, info = orc.lgmres(A, orc.PC(A, "ilu0"), b, restart=10, aug_k=3, rtol=1e-10)
    assert info["status"] == 0
    assert np.linalg.norm(b - S @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001


def _block_chain(nb, bs, seed):
    """Block-tridiagonal, block diagonally dominant matrix (1-D chain of blocks)."""
    rng = np.random.default_rng(seed)
    ptr, col, val = [0], [], []
    for I in range(nb):
        for J in (I - 1, I, I + 1):
            if 0 <= J < nb:
                B = -0.3 * rng.random((bs, bs))
                if I == J:
                    B = B + 4.0 * np.eye(bs)
                col.append(J)
                val.append(B)
        ptr.append(len(col))
    return dict(nb=nb, bs=bs, browptr=np.array(ptr, np.int32), bcol=np.array(col, np.int32),
                bval=np.array(val).reshape(-1))


def test_block_ras_special_cases(orc):
    nb, bs = 30, 3
    m = _block_chain(nb, bs, 100)
    A = orc.Mat.bsr(m)
    D = sp.bsr_matrix((m["bval"].reshape(-1, bs, bs), m["bcol"], m["browptr"]), shape=(nb * bs, nb * bs)).toarray()
    r = np.random.default_rng(101).standard_normal(nb * bs)
    # one subdomain without overlap is block ILU(0), bit for bit
    _, _, blu, bdinv = orc.bilu0(A)
    assert np.array_equal(orc.Ras(A, 1, overlap=0).apply(r), orc.bilu0_solve(A, blu, bdinv, r))
    # on a block chain every local block ILU(0) is an exact block LU: RAS is the
    # restricted dense solve on each extended set of blocks
    part = np.random.default_rng(102).integers(0, 4, nb).astype(np.int32)
    P = np.zeros((nb, nb), dtype=bool)
    for I in range(nb):
        P[I, m["bcol"][m["browptr"][I]:m["browptr"][I + 1]]] = True
    for overlap in (0, 1, 2):
        z = orc.Ras(A, 4, part=part, overlap=overlap).apply(r)
        want = np.empty(nb * bs)
        for s in range(4):
            e = part == s
            for _ in range(overlap):
                e = e | P[e].any(axis=0)
            blocks = np.nonzero(e)[0]
            if blocks.size == 0:
                continue
            idx = (blocks[:, None] * bs + np.arange(bs)).reshape(-1)
            ze = np.linalg.solve(D[np.ix_(idx, idx)], r[idx])
            own = np.repeat(part[blocks] == s, bs)
            want[idx[own]] = ze[own]
        assert np.allclose(z, want, rtol=1e-13, atol=1e-13), overlap


def test_cpr_with_ras_f_stage_is_the_composition(orc):
    # CPR-PF with R(A)^{-1} = RAS: z1 = Pi_p ILU0(App')^{-1} Pi_r f,
    # t = f - A z1, z = z1 + RAS(A)^{-1} t, from the separately pinned pieces
    g = synth.Grid(7, 6, 5)
    m = synth.black_oil_bsr3(g, 103)
    A = orc.Mat.bsr(m)
    nb, bs = g.n, 3
    part = (np.arange(nb) * 3 // nb).astype(np.int32)
    ras = dict(nsub=3, part=part, overlap=1)
    f = synth.x_true(nb * bs, 103)
    M = orc.PC(A, "cpr", ras=ras)
    w = orc.qimpes_weights(A)
    App = orc.Mat(m["browptr"], m["bcol"], orc.qimpes_app(A, w), 1)
    _, _, lu = orc.ilu0(App)
    z1 = orc.prolong(nb, bs, orc.ilu0_solve(App, lu, orc.qimpes_restrict(nb, bs, w, f)))
    want = z1 + orc.Ras(A, **ras).apply(f - orc.spmv(A, z1))
    assert np.allclose(M.apply(f), want, rtol=1e-14, atol=1e-14)


# ----------------------------------------------------------------------------
# ILUT(p, tol), the other local solver of RAS (Fig. 31)
# ----------------------------------------------------------------------------
def _ilut_dense(n, ptr, col, lu):
    L, U = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for q in range(ptr[i], ptr[i + 1]):
            (L if col[q] < i else U)[i, col[q]] = lu[q]
    return L, U


def test_ilut_without_dropping_is_the_exact_lu(orc):
    rng = np.random.default_rng(110)
    n = 40
    D = np.where(rng.random((n, n)) < 0.08, -rng.random((n, n)), 0.0)
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, np.abs(D).sum(axis=1) + 1.0)
    st, _, ptr, col, lu = orc.ilut(orc.Mat.csr(csr_dict(D)), n, 0.0)
    assert st == 0
    L, U = _ilut_dense(n, ptr, col, lu)
    P, Lr, Ur = sla.lu(D)
    assert np.array_equal(P, np.eye(n))
    assert np.allclose(L, Lr, atol=1e-14) and np.allclose(U, Ur, atol=1e-13)
    assert ptr[-1] > csr_dict(D)["col"].size            # the fill was kept


def test_ilut_special_cases(orc):
    d = synth.pressure_7pt(synth.Grid(6, 5, 4), 111)
    n = d["n"]
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(n, n)).toarray()
    # every multiplier below a huge threshold: no elimination, no off-diagonal: Jacobi
    st, _, ptr, col, lu = orc.ilut(A, 5, 1e30)
    assert st == 0 and np.array_equal(col, np.arange(n)) and np.array_equal(lu, np.diag(S))
    # a first row has nothing to eliminate: its U part keeps exactly its p largest entries
    row = np.array([5.0, -0.5, 0.0, -2.0, 0.0, -1.0, -3.0, 0.0])
    D = np.diag(np.full(8, 10.0))
    D[0] = row
    st, _, ptr, col, lu = orc.ilut(orc.Mat.csr(csr_dict(D)), 2, 0.0)
    assert st == 0 and list(col[ptr[0]:ptr[1]]) == [0, 3, 6] and list(lu[ptr[0]:ptr[1]]) == [5.0, -2.0, -3.0]
    # the dropping rule on a 3-D problem: kept entries reach tol ||a_i||, at most p per part
    tol, p = 0.05, 2
    st, _, ptr, col, lu = orc.ilut(A, p, tol)
    assert st == 0
    for i in range(n):
        c, v = col[ptr[i]:ptr[i + 1]], lu[ptr[i]:ptr[i + 1]]
        assert (np.diff(c) > 0).all() and i in c
        off = c != i
        assert (np.abs(v[off]) >= tol * np.linalg.norm(S[i])).all()
        assert (c < i).sum() <= p and (c > i).sum() <= p
    # a chain: ILUT without dropping is the exact LU (the Thomas algorithm)
    d1 = csr_dict(poisson1d(30))
    st, _, ptr, col, lu = orc.ilut(orc.Mat.csr(d1), -1, 0.0)
    L, U = _ilut_dense(30, ptr, col, lu)
    assert np.allclose(L @ U, poisson1d(30).toarray(), atol=1e-14)


def test_ras_with_ilut_local_solvers(orc):
    d = synth.pressure_7pt(synth.Grid(12, 10, 8), 112, kz_scale=0.1)
    A = orc.Mat.csr(d)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]))
    r = synth.x_true(d["n"], 112)
    # one subdomain without overlap is global ILUT
    st, _, ptr, col, lu = orc.ilut(A, -1, 1e-3)
    R = orc.Ras(A, 1, overlap=0, ilut=(-1, 1e-3))
    gidx, ptr2, col2, lu2 = R.structure()
    assert np.array_equal(ptr, ptr2) and np.array_equal(col, col2) and np.array_equal(lu, lu2)
    # RAS with ILUT local solvers preconditions GMRES
    b = S @ r
    M = orc.PC(A, "ras", ras=dict(nsub=8, overlap=1, ilut=(-1, 1e-3)))
    x, info, _ = orc.gmres(A, M, b, restart=30, rtol=1e-10)
    assert info["status"] == 0
    assert np.linalg.norm(b - S @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001
    assert orc.Ras(A, 2, ilut=(-1, -1.0)).status == orc.INVALID
