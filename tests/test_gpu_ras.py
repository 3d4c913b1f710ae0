"""Restricted additive Schwarz (Sec. 4.1) on the GPU against the CPU oracle,
through the C ABI.

The stacked extended subdomains (global row of every stacked row, pattern)
must match the oracle's bit for bit; factors within 1e-10 relative, applies
within 1e-12 relative; GMRES iteration counts within 2 of the oracle's, true
relative residual <= 1e-8 and solution within 1e-6 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(rs):
    return rs.Context(0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _partition(rs, orc, kind, g, nparts, seed=0):
    if kind == "rows":
        return None, nparts                       # contiguous ranges of rows
    if kind == "box":
        part = rs.box_partition((g.nx, g.ny, g.nz), nparts)
        return part, int(np.prod(nparts))
    rng = np.random.default_rng(seed)             # scattered, ragged subdomains
    return rng.integers(0, nparts, g.n).astype(np.int32), nparts


CASES = [
    ((6, 5, 4), "rows", 1, 0, 0),
    ((24, 20, 17), "rows", 5, 1, 0),
    ((24, 20, 17), "box", (2, 2, 2), 1, 1),
    ((32, 32, 32), "box", (2, 2, 2), 2, 0),
    ((33, 17, 9), "random", 7, 1, 1),
    ((20, 12, 8), "rows", 1920, 0, 0),            # one row per subdomain
]


@pytest.mark.parametrize("shape,kind,nparts,overlap,level", CASES)
def test_ras_structure_factors_apply(rs, ctx, orc, shape, kind, nparts, overlap, level):
    g = synth.Grid(*shape)
    d = synth.pressure_7pt(g, 50, kz_scale=0.1)
    part, np_ = _partition(rs, orc, kind, g, nparts)
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "ras", nparts=np_, part=part, overlap=overlap, level=level)
    Ao = orc.Mat.csr(d)
    R = orc.Ras(Ao, np_, part=part, overlap=overlap, level=level)
    assert R.status == 0
    gidx, ptr, col, lu = M.ras_structure()
    ogidx, optr, ocol, olu = R.structure()
    assert np.array_equal(gidx, ogidx) and np.array_equal(ptr, optr) and np.array_equal(col, ocol)
    assert np.max(np.abs(lu - olu) / np.maximum(np.abs(olu), 1e-300)) <= 1e-10
    r = np.random.default_rng(51).standard_normal(g.n)
    z = rs.Vec.zeros(ctx, g.n)
    M.apply(rs.Vec(ctx, r), z)
    zref = R.apply(r)
    assert rel(z.numpy(), zref) <= 1e-12
    z2 = rs.Vec.zeros(ctx, g.n)
    for _ in range(2):                            # the sweep state cleans itself
        M.apply(rs.Vec(ctx, r), z2)
    assert np.array_equal(z.numpy(), z2.numpy())
    Mm = rs.Precond(ctx, A, "ras", prec="mixed", nparts=np_, part=part, overlap=overlap, level=level)
    Mm.apply(rs.Vec(ctx, r), z2)
    assert rel(z2.numpy(), zref) <= 1e-5


@pytest.mark.parametrize("solver", ["gmres", "bicgstab"])
@pytest.mark.parametrize("shape,kz,parts,overlap,level", [
    ((32, 32, 32), 1.0, (2, 2, 2), 1, 0),
    ((20, 17, 9), 0.1, (3, 2, 1), 1, 1),
    ((24, 24, 24), 1.0, (4, 4, 4), 0, 0),
])
def test_ras_krylov_parity(rs, ctx, orc, solver, shape, kz, parts, overlap, level):
    g = synth.Grid(*shape)
    d = synth.pressure_7pt(g, 52, kz_scale=kz)
    part = rs.box_partition(shape, parts)
    nparts = int(np.prod(parts))
    Ao = orc.Mat.csr(d)
    b = orc.spmv(Ao, synth.x_true(g.n, 52))
    Mo = orc.PC(Ao, "ras", ras=dict(nsub=nparts, part=part, overlap=overlap, level=level))
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "ras", nparts=nparts, part=part, overlap=overlap, level=level)
    x = rs.Vec.zeros(ctx, g.n)
    if solver == "gmres":
        xo, io, _ = orc.gmres(Ao, Mo, b, restart=30, rtol=1e-8)
        info = rs.solve_gmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8, maxit=10000)
    else:
        xo, io, _ = orc.bicgstab(Ao, Mo, b, rtol=1e-8)
        info = rs.solve_bicgstab(A, M, rs.Vec(ctx, b), x, rtol=1e-8, maxit=10000)
    xs = x.numpy()
    true = orc.norm2(b - orc.spmv(Ao, xs)) / orc.norm2(b)
    assert info["status"] == 0 and io["status"] == 0
    assert true <= 1e-8
    if solver == "gmres":
        assert abs(info["iters"] - io["iters"]) <= 2, (info, io)
        assert rel(xs, xo) <= 1e-6
    else:
        # BiCGSTAB's first crossing of rtol moves with rounding; both meet it
        lo = orc.bicgstab(Ao, Mo, b, rtol=2e-8)[1]["iters"]
        hi = orc.bicgstab(Ao, Mo, b, rtol=5e-9)[1]["iters"]
        assert min(lo, hi, io["iters"]) - 2 <= info["iters"] <= max(lo, hi, io["iters"]) + 2, (info, io)


def test_ras_block_matrix(rs, ctx, orc):
    """Block rows of a BSR matrix as subdomains, block ILU(0) local solver:
    the reference is the oracle's block ILU(0) on each extended block set,
    restricted to the owned block rows."""
    g = synth.Grid(9, 7, 5)
    m = synth.black_oil_bsr3(g, 53)
    nb, bs = g.n, 3
    part = rs.box_partition((g.nx, g.ny, g.nz), (2, 2, 1))
    A = rs.Mat.bsr(ctx, m)
    r = np.random.default_rng(54).standard_normal(nb * bs)
    P = sp.csr_matrix((np.ones(m["bcol"].size), m["bcol"], m["browptr"]), shape=(nb, nb)).toarray() != 0
    B = m["bval"].reshape(-1, bs, bs)
    for overlap in (0, 1):
        M = rs.Precond(ctx, A, "ras", nparts=4, part=part, overlap=overlap)
        z = rs.Vec.zeros(ctx, nb * bs)
        M.apply(rs.Vec(ctx, r), z)
        want = np.empty(nb * bs)
        for s in range(4):
            e = part == s
            for _ in range(overlap):
                e = e | P[e].any(axis=0)
            rows = np.nonzero(e)[0]
            loc = -np.ones(nb, np.int64)
            loc[rows] = np.arange(rows.size)
            ptr, col, val = [0], [], []
            for I in rows:
                for q in range(m["browptr"][I], m["browptr"][I + 1]):
                    J = m["bcol"][q]
                    if loc[J] >= 0:
                        col.append(loc[J])
                        val.append(B[q])
                ptr.append(len(col))
            sub = dict(nb=rows.size, bs=bs, browptr=np.array(ptr, np.int32), bcol=np.array(col, np.int32),
                       bval=np.array(val).reshape(-1))
            Ao = orc.Mat.bsr(sub)
            st, _, blu, bdinv = orc.bilu0(Ao)
            assert st == 0
            idx = (rows[:, None] * bs + np.arange(bs)).reshape(-1)
            zs = orc.bilu0_solve(Ao, blu, bdinv, r[idx])
            own = np.repeat(part[rows] == s, bs)
            want[idx[own]] = zs[own]
        assert rel(z.numpy(), want) <= 1e-12, overlap


def test_ras_sweep_levels_shrink_with_subdomains(rs, ctx):
    g = synth.Grid(64, 64, 32)
    d = synth.pressure_7pt(g, 55)
    A = rs.Mat.csr(ctx, d)
    l0, u0 = rs.Precond(ctx, A, "ilu0", sweep="segments").sweep_levels()
    M = rs.Precond(ctx, A, "ras", nparts=32, part=rs.box_partition((64, 64, 32), (4, 4, 2)), overlap=1)
    l1, u1 = M.sweep_levels()
    # one subdomain of 16 x 16 x 16 cells plus one layer: at most 1 + 18 + 18 - 2 segment levels
    assert l1 <= 35 and u1 <= 35 and l1 < l0 / 2 and u1 < u0 / 2, (l0, u0, l1, u1)


def test_ras_invalid_arguments(rs, ctx):
    g = synth.Grid(6, 5, 4)
    A = rs.Mat.csr(ctx, synth.pressure_7pt(g, 56))
    bad = [dict(nparts=-1), dict(nparts=2, part=np.full(g.n, 2, np.int32)), dict(nparts=2, overlap=-1),
           dict(nparts=2, level=9), dict(nparts=2, part=np.full(g.n, -1, np.int32))]
    for kw in bad:
        with pytest.raises(rs.RsError) as e:
            rs.Precond(ctx, A, "ras", **kw)
        assert e.value.status == rs.ERR_INVALID_ARG, kw


@pytest.mark.parametrize("form,pstage", [("pf", "ilu0"), ("fpf", "ilu0"), ("fpf", "amg")])
def test_cpr_with_ras_f_stage(rs, ctx, orc, form, pstage):
    """CPR whose F stage R(A)^{-1} is RAS over block subdomains (the paper's
    CPR arrangement, Sec. 4.2.1), against the oracle's."""
    g = synth.Grid(11, 9, 7)
    m = synth.black_oil_bsr3(g, 57)
    part = rs.box_partition((g.nx, g.ny, g.nz), (2, 2, 1))
    Ao = orc.Mat.bsr(m)
    kw = dict(amg=dict()) if pstage == "amg" else {}
    Mo = orc.PC(Ao, "cpr", form=form, ras=dict(nsub=4, part=part, overlap=1), **kw)
    A = rs.Mat.bsr(ctx, m)
    M = rs.Precond(ctx, A, "cpr", form=form, nparts=4, part=part, overlap=1, pstage=pstage)
    r = np.random.default_rng(58).standard_normal(A.n)
    z = rs.Vec.zeros(ctx, A.n)
    M.apply(rs.Vec(ctx, r), z)
    assert rel(z.numpy(), Mo.apply(r)) <= 1e-12
    b = orc.spmv(Ao, synth.x_true(A.n, 58))
    xo, io, _ = orc.gmres(Ao, Mo, b, restart=30, rtol=1e-8, flexible=True)
    x = rs.Vec.zeros(ctx, A.n)
    info = rs.solve_fgmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8, maxit=10000)
    assert info["status"] == 0 and io["status"] == 0 and info["true_rel_res"] <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= 2, (info, io)


def test_ras_degenerate_cases(rs, ctx, orc):
    g = synth.Grid(7, 6, 5)
    d = synth.pressure_7pt(g, 59)
    A = rs.Mat.csr(ctx, d)
    Ao = orc.Mat.csr(d)
    r = np.random.default_rng(60).standard_normal(g.n)
    # more subdomains than used: empty parts are skipped
    part = (np.arange(g.n) % 5 * 2).astype(np.int32)            # parts 0, 2, 4, 6, 8 of 10
    for overlap in (0, 1):
        M = rs.Precond(ctx, A, "ras", nparts=10, part=part, overlap=overlap)
        z = rs.Vec.zeros(ctx, g.n)
        M.apply(rs.Vec(ctx, r), z)
        assert rel(z.numpy(), orc.Ras(Ao, 10, part=part, overlap=overlap).apply(r)) <= 1e-12
    # overlap beyond the graph's diameter: every subdomain is the whole matrix,
    # so every row takes the global ILU(0) solution
    M = rs.Precond(ctx, A, "ras", nparts=3, overlap=50)
    z = rs.Vec.zeros(ctx, g.n)
    M.apply(rs.Vec(ctx, r), z)
    _, _, lu = orc.ilu0(Ao)
    assert rel(z.numpy(), orc.ilu0_solve(Ao, lu, r)) <= 1e-12
    # a 1 x 1 system
    one = dict(n=1, rowptr=np.array([0, 1], np.int32), col=np.array([0], np.int32), val=np.array([4.0]))
    M1 = rs.Precond(ctx, rs.Mat.csr(ctx, one), "ras", nparts=1, overlap=1, level=1)
    z1 = rs.Vec.zeros(ctx, 1)
    M1.apply(rs.Vec(ctx, np.array([2.0])), z1)
    assert z1.numpy()[0] == 0.5


def test_cpr_ras_f_stage_on_a_scalar_matrix(rs, ctx, orc):
    g = synth.Grid(10, 8, 6)
    d = synth.pressure_7pt(g, 61, kz_scale=0.1)
    part = rs.box_partition((g.nx, g.ny, g.nz), (2, 2, 2))
    Ao = orc.Mat.csr(d)
    Mo = orc.PC(Ao, "cpr", ras=dict(nsub=8, part=part, overlap=1))
    M = rs.Precond(ctx, rs.Mat.csr(ctx, d), "cpr", nparts=8, part=part, overlap=1)
    r = np.random.default_rng(62).standard_normal(g.n)
    z = rs.Vec.zeros(ctx, g.n)
    M.apply(rs.Vec(ctx, r), z)
    assert rel(z.numpy(), Mo.apply(r)) <= 1e-12


@pytest.mark.parametrize("shape,parts,overlap,ilut", [
    ((20, 16, 12), (2, 2, 2), 1, (-1, 1e-3)),
    ((24, 20, 17), (3, 2, 1), 2, (3, 1e-2)),
    ((16, 16, 16), (1, 1, 1), 0, (-1, 1e-4)),
    # nothing dropped: complete fill, several times the first output region,
    # so the factorisation is repeated with doubled regions
    ((10, 9, 8), (2, 1, 1), 1, (1000, 1e-300)),
])
def test_ras_ilut_parity(rs, ctx, orc, shape, parts, overlap, ilut):
    g = synth.Grid(*shape)
    d = synth.pressure_7pt(g, 63, kz_scale=0.1)
    part = rs.box_partition(shape, parts)
    nparts = int(np.prod(parts))
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "ras", nparts=nparts, part=part, overlap=overlap, ilut=ilut)
    Ao = orc.Mat.csr(d)
    R = orc.Ras(Ao, nparts, part=part, overlap=overlap, ilut=ilut)
    assert R.status == 0
    gidx, ptr, col, lu = M.ras_structure()
    ogidx, optr, ocol, olu = R.structure()
    # the dropping decisions agree, so the patterns are identical
    assert np.array_equal(gidx, ogidx) and np.array_equal(ptr, optr) and np.array_equal(col, ocol)
    assert np.max(np.abs(lu - olu) / np.maximum(np.abs(olu), 1e-300)) <= 1e-12
    r = np.random.default_rng(64).standard_normal(g.n)
    z = rs.Vec.zeros(ctx, g.n)
    M.apply(rs.Vec(ctx, r), z)
    assert rel(z.numpy(), R.apply(r)) <= 1e-12
    b = orc.spmv(Ao, synth.x_true(g.n, 64))
    Mo = orc.PC(Ao, "ras", ras=dict(nsub=nparts, part=part, overlap=overlap, ilut=ilut))
    xo, io, _ = orc.gmres(Ao, Mo, b, restart=30, rtol=1e-8)
    x = rs.Vec.zeros(ctx, g.n)
    info = rs.solve_gmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8, maxit=10000)
    assert info["status"] == 0 and io["status"] == 0 and info["true_rel_res"] <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= 2, (info, io)


def test_ras_ilut_zero_pivot_reports_the_global_row(rs, ctx, orc):
    """Subdomain 1 holds rows 1 and 2 without overlap; its local row 1 has the
    pivot 1 - 1 * 1 = 0, so ILUT stops there and reports global row 2."""
    d = dict(n=3, rowptr=np.array([0, 2, 5, 7], np.int32), col=np.array([0, 1, 0, 1, 2, 1, 2], np.int32),
             val=np.array([1.0, 2.0, 0.5, 1.0, 1.0, 1.0, 1.0]))
    part = np.array([0, 1, 1], np.int32)
    R = orc.Ras(orc.Mat.csr(d), 2, part=part, overlap=0, ilut=(-1, 1e-3))
    assert R.status != 0
    M = rs.Precond(ctx, rs.Mat.csr(ctx, d), "ras", nparts=2, part=part, overlap=0, ilut=(-1, 1e-3))
    assert M.status == rs.ERR_ZERO_PIVOT and M.bad_row == 2


def test_ras_ilut_rejected_on_blocks(rs, ctx):
    m = synth.black_oil_bsr3(synth.Grid(6, 5, 4), 65)
    with pytest.raises(rs.RsError) as e:
        rs.Precond(ctx, rs.Mat.bsr(ctx, m), "ras", nparts=2, ilut=(-1, 1e-3))
    assert e.value.status == rs.ERR_INVALID_ARG
