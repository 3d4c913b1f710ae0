"""Algebraic multigrid (Sec. 4.2, Algs. 3-4) on the GPU against the CPU
oracle, through the C ABI.

The hierarchy is built on the GPU (strength, PMIS coarsening with the
SplitMix64 weights, direct interpolation, Galerkin products) and must match
the oracle's bit for bit: the C/F splitting, the patterns and the values of
every A_l and P_l (both sides sum every entry's terms in the same order,
each product and sum rounded once).  The V-cycle apply within 1e-12 relative, with
either smoother; PCG /
GMRES with AMG within 2 iterations of the oracle, true relative residual
<= 1e-8, solution within 1e-6 relative.  The test matrices have random
coefficients so that no strength comparison sits exactly on the threshold.
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


def relmax(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300) if b.size else 0.0


def _poisson1d(n):
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    A.sort_indices()
    return dict(n=n, rowptr=A.indptr.astype(np.int32), col=A.indices.astype(np.int32), val=A.data.copy())


PROBLEMS = [
    ("7pt", (24, 20, 17), 0.1, dict()),
    ("7pt", (32, 32, 32), 1.0, dict()),
    ("7pt", (40, 9, 5), 1.0, dict(max_coarse=5, nu=1)),
    ("1d", (63,), None, dict(max_coarse=1)),                 # dyadic values: exact on both sides
    ("7pt", (16, 16, 16), 1.0, dict(theta=0.25, max_levels=3)),
]


def _matrix(kind, shape, kz, seed=70):
    if kind == "1d":
        return _poisson1d(shape[0])
    return synth.pressure_7pt(synth.Grid(*shape), seed, kz_scale=kz)


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("kind,shape,kz,kw", PROBLEMS)
def test_amg_hierarchy_and_vcycle(rs, ctx, orc, kind, shape, kz, kw, smoother):
    """smoother 0: l1-Jacobi; 1: hybrid Gauss-Seidel over 32-row chunks
    (Fig. 34's relaxation), forward before and backward after the coarse
    correction."""
    d = _matrix(kind, shape, kz)
    n = d["n"]
    kw = dict(kw, smoother=smoother)
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "amg", amg=kw)
    R = orc.Amg(orc.Mat.csr(d), **kw)
    assert R.status == 0
    got, want = M.amg_levels(), R.levels()
    assert len(got) == len(want) >= 2
    for l, (g, (wa, wp)) in enumerate(zip(got, want)):
        assert np.array_equal(g["A"][0], wa[0]) and np.array_equal(g["A"][1], wa[1]), l
        assert np.array_equal(g["A"][2], wa[2]), (l, relmax(g["A"][2], wa[2]))
        if wp is not None:
            assert np.array_equal(g["cidx"], R.cidx(l)), l
            assert np.array_equal(g["P"][0], wp[0]) and np.array_equal(g["P"][1], wp[1]), l
            assert np.array_equal(g["P"][2], wp[2]), (l, relmax(g["P"][2], wp[2]))
    r = np.random.default_rng(71).standard_normal(n)
    z = rs.Vec.zeros(ctx, n)
    M.apply(rs.Vec(ctx, r), z)
    zref = R.apply(r)
    assert rel(z.numpy(), zref) <= 1e-12
    z2 = rs.Vec.zeros(ctx, n)
    M.apply(rs.Vec(ctx, r), z2)
    assert np.array_equal(z.numpy(), z2.numpy())


def test_amg_setup_at_full_size(rs, ctx, orc):
    """The GPU setup at 128 x 128 x 64 (8 levels): the C/F splitting of every
    level, the patterns and values of every A_l and P_l equal the oracle's."""
    g = synth.Grid(128, 128, 64)
    d = synth.pressure_7pt(g, 1, kz_scale=0.1)
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "amg")
    R = orc.Amg(orc.Mat.csr(d))
    got, want = M.amg_levels(), R.levels()
    assert len(got) == len(want) >= 5
    for l, (gl, (wa, wp)) in enumerate(zip(got, want)):
        assert all(np.array_equal(x, y) for x, y in zip(gl["A"], wa)), l
        if wp is not None:
            assert np.array_equal(gl["cidx"], R.cidx(l)), l
            assert all(np.array_equal(x, y) for x, y in zip(gl["P"], wp)), l


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("solver", ["cg", "gmres"])
@pytest.mark.parametrize("shape,kz", [((32, 32, 32), 1.0), ((30, 22, 13), 0.1)])
def test_amg_krylov_parity(rs, ctx, orc, solver, shape, kz, smoother):
    g = synth.Grid(*shape)
    d = synth.pressure_7pt(g, 72, kz_scale=kz)
    Ao = orc.Mat.csr(d)
    b = orc.spmv(Ao, synth.x_true(g.n, 72))
    Mo = orc.PC(Ao, "amg", amg=dict(smoother=smoother))
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "amg", amg=dict(smoother=smoother))
    x = rs.Vec.zeros(ctx, g.n)
    if solver == "cg":
        xo, io, _ = orc.cg(Ao, Mo, b, rtol=1e-8)
        info = rs.solve_cg(A, M, rs.Vec(ctx, b), x, rtol=1e-8, maxit=10000)
    else:
        xo, io, _ = orc.gmres(Ao, Mo, b, restart=30, rtol=1e-8)
        info = rs.solve_gmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8, maxit=10000)
    xs = x.numpy()
    true = orc.norm2(b - orc.spmv(Ao, xs)) / orc.norm2(b)
    assert info["status"] == 0 and io["status"] == 0
    assert true <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= 2, (info, io)
    assert rel(xs, xo) <= 1e-6


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("form", ["pf", "fpf"])
def test_cpr_amg_pressure_stage(rs, ctx, orc, form, smoother):
    g = synth.Grid(14, 12, 9)
    m = synth.black_oil_bsr3(g, 73)
    Ao = orc.Mat.bsr(m)
    Mo = orc.PC(Ao, "cpr", form=form, amg=dict(smoother=smoother))
    A = rs.Mat.bsr(ctx, m)
    M = rs.Precond(ctx, A, "cpr", form=form, pstage="amg", amg=dict(smoother=smoother))
    r = np.random.default_rng(74).standard_normal(A.n)
    z = rs.Vec.zeros(ctx, A.n)
    M.apply(rs.Vec(ctx, r), z)
    assert rel(z.numpy(), Mo.apply(r)) <= 1e-12
    b = orc.spmv(Ao, synth.x_true(A.n, 74))
    xo, io, _ = orc.gmres(Ao, Mo, b, restart=30, rtol=1e-8, flexible=True)
    x = rs.Vec.zeros(ctx, A.n)
    info = rs.solve_fgmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8, maxit=10000)
    assert info["status"] == 0 and io["status"] == 0 and info["true_rel_res"] <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= 2, (info, io)


def test_amg_invalid_arguments(rs, ctx):
    g = synth.Grid(8, 7, 6)
    A = rs.Mat.csr(ctx, synth.pressure_7pt(g, 75))
    for kw in (dict(theta=1.5), dict(theta=-0.1), dict(max_levels=17), dict(nu=-1), dict(max_coarse=-3),
               dict(smoother=2), dict(smoother=-1)):
        with pytest.raises(rs.RsError) as e:
            rs.Precond(ctx, A, "amg", amg=kw)
        assert e.value.status == rs.ERR_INVALID_ARG, kw
    B = rs.Mat.bsr(ctx, synth.black_oil_bsr3(g, 75))
    with pytest.raises(rs.RsError) as e:
        rs.Precond(ctx, B, "amg")
    assert e.value.status == rs.ERR_INVALID_ARG
    # Gauss-Seidel needs a nonzero diagonal on every smoothed level
    d = _poisson1d(40)
    dz = dict(d, val=d["val"].copy())
    dz["val"][d["rowptr"][7] + 1] = 0.0             # a_77 = 0 (row 7: entries 6, 7, 8)
    Z = rs.Mat.csr(ctx, dz)
    Mz = rs.Precond(ctx, Z, "amg", amg=dict(smoother=1, max_coarse=4))
    assert Mz.status == rs.ERR_ZERO_PIVOT and not Mz.h    # no hierarchy, no handle
    with pytest.raises(rs.RsError):
        Mz.apply(rs.Vec.zeros(ctx, 40), rs.Vec.zeros(ctx, 40))
    assert rs.Precond(ctx, Z, "amg", amg=dict(smoother=0, max_coarse=4)).status == rs.OK


def test_amg_degenerate_cases(rs, ctx, orc):
    # below max_coarse: one level, the V-cycle is the dense solve
    g = synth.Grid(6, 5, 4)
    d = synth.pressure_7pt(g, 76)
    A = rs.Mat.csr(ctx, d)
    M = rs.Precond(ctx, A, "amg")
    assert len(M.amg_sizes()) == 1
    r = np.random.default_rng(77).standard_normal(g.n)
    z = rs.Vec.zeros(ctx, g.n)
    M.apply(rs.Vec(ctx, r), z)
    S = sp.csr_matrix((d["val"], d["col"], d["rowptr"]), shape=(g.n, g.n)).toarray()
    assert rel(z.numpy(), np.linalg.solve(S, r)) <= 1e-12
    # a diagonal matrix has no strong connections: no coarse points.  Up to
    # 4096 rows the single level is solved densely; above, setup refuses it
    for n, ok in ((3000, True), (5000, False)):
        dg = dict(n=n, rowptr=np.arange(n + 1, dtype=np.int32), col=np.arange(n, dtype=np.int32),
                  val=1.0 + np.arange(n, dtype=float))
        D = rs.Mat.csr(ctx, dg)
        if ok:
            Md = rs.Precond(ctx, D, "amg")
            rr = np.random.default_rng(78).standard_normal(n)
            zz = rs.Vec.zeros(ctx, n)
            Md.apply(rs.Vec(ctx, rr), zz)
            assert rel(zz.numpy(), rr / dg["val"]) <= 1e-14
        else:
            with pytest.raises(rs.RsError) as e:
                rs.Precond(ctx, D, "amg")
            assert e.value.status == rs.ERR_INVALID_ARG
