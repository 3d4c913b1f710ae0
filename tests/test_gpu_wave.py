"""Wavefront triangular sweeps (ILU(0) and block ILU(0) on structured
7-point grids, Eq. 3) against the CPU oracle and against the segment
sweeps, through the C ABI.

The shapes cover several units per plane with a partial last one (ny not a
multiple of 32), x-lines shorter than a warp, planes of one unit, two-
dimensional grids, patterns with entries knocked out (a subset of the
stencil), and the benchmarked sizes.  Tolerances: FP64 within 1e-12 of the
oracle's solve, FP32 within 1e-5 of the oracle's FP32 solve.
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


SHAPES = [(5, 4, 3), (24, 20, 17), (33, 70, 5), (7, 33, 4), (100, 100, 3), (128, 40, 2), (3, 65, 6), (64, 64, 1)]


@pytest.mark.parametrize("shape", SHAPES)
def test_wave_ilu0_apply_matches_oracle_and_segments(rs, ctx, orc, shape):
    g = synth.Grid(*shape)
    d = synth.pressure_7pt(g, 31, kz_scale=0.1)
    A = rs.Mat.csr(ctx, d)
    Ao = orc.Mat.csr(d)
    _, _, lu = orc.ilu0(Ao)
    r = np.random.default_rng(32).standard_normal(g.n)
    nx, ny, nz = shape
    for prec in ("fp64", "mixed"):
        W = rs.Precond(ctx, A, "ilu0", prec=prec, sweep="wavefront")
        # a 2-D grid reads as nx x ny x 1; a grid with ny = 1 as nx x nz x 1
        assert W.sweep_kind() == ("wavefront", (nx, ny, nz))
        assert np.array_equal(W.ilu_factors(d["col"].size), lu)
        S = rs.Precond(ctx, A, "ilu0", prec=prec, sweep="segments")
        ref = orc.ilu0_solve(Ao, lu, r, fp32=(prec == "mixed"))
        tol = 1e-12 if prec == "fp64" else 1e-5
        zw, zs = rs.Vec.zeros(ctx, g.n), rs.Vec.zeros(ctx, g.n)
        for _ in range(3):     # the work vectors return to the sentinel between applies
            W.apply(rs.Vec(ctx, r), zw)
            assert rel(zw.numpy(), ref) <= tol
        S.apply(rs.Vec(ctx, r), zs)
        assert rel(zw.numpy(), zs.numpy()) <= 2 * tol


def test_wave_is_bit_stable_across_applies_and_scales(rs, ctx, orc):
    """The schedule is dynamic (tickets), the arithmetic is not: repeated
    applies give identical bits; a device scale multiplies r on entry."""
    g = synth.Grid(40, 50, 12)
    d = synth.pressure_7pt(g, 41)
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "ilu0", sweep="wavefront")
    r = np.random.default_rng(42).standard_normal(g.n)
    z1, z2 = rs.Vec.zeros(ctx, g.n), rs.Vec.zeros(ctx, g.n)
    M.apply(rs.Vec(ctx, r), z1)
    for _ in range(5):
        M.apply(rs.Vec(ctx, r), z2)
        assert np.array_equal(z1.numpy(), z2.numpy())


@pytest.mark.parametrize("drop,seed", [(0.1, 1), (0.4, 2)])
def test_wave_subset_pattern(rs, ctx, orc, drop, seed):
    """Off-diagonal entries knocked out at random (a subset of the 7-point
    stencil, not symmetric): still a grid pattern, and ILU(0) keeps it."""
    g = synth.Grid(30, 45, 7)
    d = synth.pressure_7pt(g, 50 + seed)
    M0 = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(g.n, g.n)).tocoo()
    rng = np.random.default_rng(seed)
    keep = (M0.row == M0.col) | (rng.random(M0.nnz) > drop)
    B = sp.csr_matrix((M0.data[keep], (M0.row[keep], M0.col[keep])), shape=M0.shape)
    B.sort_indices()
    dd = dict(n=g.n, rowptr=B.indptr.astype(np.int32), col=B.indices.astype(np.int32), val=B.data.copy())
    A = rs.Mat.csr(ctx, dd)
    Ao = orc.Mat.csr(dd)
    st, _, lu = orc.ilu0(Ao)
    assert st == 0
    r = rng.standard_normal(g.n)
    for prec in ("fp64", "mixed"):
        M = rs.Precond(ctx, A, "ilu0", prec=prec, sweep="wavefront")
        assert M.sweep_kind()[0] == "wavefront"
        z = rs.Vec.zeros(ctx, g.n)
        M.apply(rs.Vec(ctx, r), z)
        assert rel(z.numpy(), orc.ilu0_solve(Ao, lu, r, fp32=(prec == "mixed"))) <= (1e-12 if prec == "fp64" else 1e-5)


def test_library_choice_is_the_wavefront_on_grids(rs, ctx):
    """The default sweep option takes the wavefront sweeps on a structured
    7-point pattern (scalar and block) and the segment sweeps elsewhere."""
    g = synth.Grid(20, 12, 6)
    A = rs.Mat.csr(ctx, synth.pressure_7pt(g, 60))
    assert rs.Precond(ctx, A, "ilu0").sweep_kind() == ("wavefront", (20, 12, 6))
    assert rs.Precond(ctx, A, "ilu0", sweep="segments").sweep_kind() == ("segments", None)
    B = rs.Mat.bsr(ctx, synth.black_oil_bsr3(g, 61))
    assert rs.Precond(ctx, B, "bilu0").sweep_kind() == ("wavefront", (20, 12, 6))
    n = 300
    D = sp.random(n, n, density=0.02, random_state=7, format="csr") * -1.0
    D = (D + sp.diags(np.abs(D).sum(axis=1).A1 + 1.0)).tocsr()
    D.sort_indices()
    d = dict(n=n, rowptr=D.indptr.astype(np.int32), col=D.indices.astype(np.int32), val=D.data.copy())
    assert rs.Precond(ctx, rs.Mat.csr(ctx, d), "ilu0").sweep_kind() == ("segments", None)


def test_non_grid_patterns_take_the_segment_sweeps(rs, ctx, orc):
    """A pattern that is not a 7-point grid (a random one; a 1-D chain; a
    27-point-like extra diagonal) keeps the segment sweeps."""
    n = 600
    D = sp.random(n, n, density=0.01, random_state=5, format="csr") * -1.0
    D = (D + sp.diags(np.abs(D).sum(axis=1).A1 + 1.0)).tocsr()
    D.sort_indices()
    d = dict(n=n, rowptr=D.indptr.astype(np.int32), col=D.indices.astype(np.int32), val=D.data.copy())
    assert rs.Precond(ctx, rs.Mat.csr(ctx, d), "ilu0", sweep="wavefront").sweep_kind() == ("segments", None)
    T = sp.diags([-np.ones(n - 1), 3 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    T.sort_indices()
    d = dict(n=n, rowptr=T.indptr.astype(np.int32), col=T.indices.astype(np.int32), val=T.data.copy())
    assert rs.Precond(ctx, rs.Mat.csr(ctx, d), "ilu0", sweep="wavefront").sweep_kind() == ("segments", None)
    g = synth.Grid(10, 9, 8)
    P = sp.csr_matrix((lambda m: (m["val"], m["col"], m["rowptr"]))(synth.pressure_7pt(g, 3)), shape=(g.n, g.n))
    P = (P + sp.diags([-0.01 * np.ones(g.n - 11), -0.01 * np.ones(g.n - 11)], [-11, 11])).tocsr()
    P.sort_indices()
    d = dict(n=g.n, rowptr=P.indptr.astype(np.int32), col=P.indices.astype(np.int32), val=P.data.copy())
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "ilu0", sweep="wavefront")
    assert M.sweep_kind() == ("segments", None)
    Ao = orc.Mat.csr(d)
    _, _, lu = orc.ilu0(Ao)
    r = np.random.default_rng(6).standard_normal(g.n)
    z = rs.Vec.zeros(ctx, g.n)
    M.apply(rs.Vec(ctx, r), z)
    assert rel(z.numpy(), orc.ilu0_solve(Ao, lu, r)) <= 1e-12


@pytest.mark.parametrize("shape", [(4, 3, 3), (13, 11, 7), (20, 40, 6), (48, 48, 32)])
def test_wave_block_ilu0_matches_oracle(rs, ctx, orc, shape):
    g = synth.Grid(*shape)
    m = synth.black_oil_bsr3(g, 8)
    A = rs.Mat.bsr(ctx, m)
    Ao = orc.Mat.bsr(m)
    st, _, lu_ref, dinv_ref = orc.bilu0(Ao)
    assert st == 0
    r = np.random.default_rng(9).standard_normal(A.n)
    for prec in ("fp64", "mixed"):
        M = rs.Precond(ctx, A, "bilu0", prec=prec, sweep="wavefront")
        assert M.sweep_kind() == ("wavefront", shape)
        S = rs.Precond(ctx, A, "bilu0", prec=prec, sweep="segments")
        ref = orc.bilu0_solve(Ao, lu_ref, dinv_ref, r, fp32=(prec == "mixed"))
        tol = 1e-12 if prec == "fp64" else 1e-5
        z, zs = rs.Vec.zeros(ctx, A.n), rs.Vec.zeros(ctx, A.n)
        for _ in range(2):
            M.apply(rs.Vec(ctx, r), z)
            assert rel(z.numpy(), ref) <= tol
        S.apply(rs.Vec(ctx, r), zs)
        assert rel(z.numpy(), zs.numpy()) <= 2 * tol


def _blocks_of_size(m3, bs):
    """The black-oil 3x3 blocks cut to their leading 2x2 (bs 2), or padded to
    4x4 with a fourth unknown coupled only to itself (bs 4, diagonal 2)."""
    b3 = m3["bval"].reshape(-1, 3, 3)
    if bs == 2:
        bv = b3[:, :2, :2]
    else:
        bv = np.zeros((b3.shape[0], 4, 4))
        bv[:, :3, :3] = b3
        row = np.repeat(np.arange(m3["nb"]), np.diff(m3["browptr"]))
        bv[row == m3["bcol"], 3, 3] = 2.0
    return dict(nb=m3["nb"], bs=bs, browptr=m3["browptr"], bcol=m3["bcol"], bval=np.ascontiguousarray(bv).reshape(-1))


@pytest.mark.parametrize("bs", [2, 4])
def test_wave_block_ilu0_other_block_sizes(rs, ctx, orc, bs):
    """2x2 and 4x4 blocks: in FP64 every block size runs its components on
    separate compute warps (2 and 4 of them), in FP32 on one."""
    shape = (13, 11, 7)
    m = _blocks_of_size(synth.black_oil_bsr3(synth.Grid(*shape), 18), bs)
    A = rs.Mat.bsr(ctx, m)
    Ao = orc.Mat.bsr(m)
    st, _, lu_ref, dinv_ref = orc.bilu0(Ao)
    assert st == 0
    r = np.random.default_rng(19).standard_normal(A.n)
    for prec in ("fp64", "mixed"):
        M = rs.Precond(ctx, A, "bilu0", prec=prec, sweep="wavefront")
        assert M.sweep_kind() == ("wavefront", shape)
        z = rs.Vec.zeros(ctx, A.n)
        M.apply(rs.Vec(ctx, r), z)
        ref = orc.bilu0_solve(Ao, lu_ref, dinv_ref, r, fp32=(prec == "mixed"))
        assert rel(z.numpy(), ref) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wave_cpr_apply_and_fgmres(rs, ctx, orc, prec):
    """CPR on the block system: both of its ILU factors (the decoupled
    pressure matrix and the block matrix) take the wavefront sweeps."""
    g = synth.Grid(16, 40, 8)
    m = synth.black_oil_bsr3(g, 21)
    Ao = orc.Mat.bsr(m)
    A = rs.Mat.bsr(ctx, m)
    M = rs.Precond(ctx, A, "cpr", prec=prec, sweep="wavefront")
    assert M.sweep_kind() == ("wavefront", (16, 40, 8))
    Mo = orc.PC(Ao, "cpr", mixed=(prec == "mixed"))
    f = np.random.default_rng(22).standard_normal(A.n)
    z = rs.Vec.zeros(ctx, A.n)
    M.apply(rs.Vec(ctx, f), z)
    assert rel(z.numpy(), Mo.apply(f)) <= (1e-12 if prec == "fp64" else 1e-5)
    b = orc.spmv(Ao, synth.x_true(Ao.n, 21))
    xo, io, _ = orc.fgmres(Ao, Mo, b, restart=30, rtol=1e-8)
    x = rs.Vec.zeros(ctx, A.n)
    info = rs.solve_fgmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8)
    assert info["status"] == 0 and abs(info["iters"] - io["iters"]) <= 2, (info, io)
    assert rel(x.numpy(), xo) <= 1e-6


def test_wave_gmres_full_size(rs, ctx, orc):
    """GMRES(30) + ILU(0) at 128 x 128 x 64 with the wavefront sweeps: the
    residual history within 1e-8 of the oracle's, equal iteration counts."""
    g = synth.Grid(128, 128, 64)
    d = synth.pressure_7pt(g, 1, kz_scale=0.1)
    Ao = orc.Mat.csr(d)
    b = orc.spmv(Ao, synth.x_true(g.n, 1))
    xo, io, ho = orc.gmres(Ao, orc.PC(Ao, "ilu0"), b, restart=30, rtol=1e-8, hist_len=4000)
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "ilu0", sweep="wavefront")
    assert M.sweep_kind() == ("wavefront", (128, 128, 64))
    hist = ctx.set_history(4000)
    x = rs.Vec.zeros(ctx, g.n)
    try:
        info = rs.solve_gmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8)
    finally:
        ctx.set_history(0)
    hs = hist[:info["iters"]]
    assert info["status"] == 0 and info["iters"] == io["iters"], (info, io)
    assert np.all(np.abs(hs - ho) <= 1e-8 * ho)
    assert rel(x.numpy(), xo) <= 1e-10
