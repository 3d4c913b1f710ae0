"""Learned pressure stage on the GPU vs the numpy oracle (oracle/convnet.py).

The CUDA path stores activations and activation gradients in bfloat16 and
accumulates in FP32; the oracle computes in FP64 and rounds activations and
weights to bfloat16 where the CUDA path stores them.  Tolerances follow from
bfloat16's 8-bit significand (relative rounding 2^-9 per stored value):
network output within 2e-2 relative (L2), each layer's weight gradient within
6e-2 relative (L2) with cosine similarity above 0.998.
"""
import os
import tempfile

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(rs):
    return rs.Context(0)


def _params(seed):
    from oracle import convnet as cn
    p = cn.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * rng.standard_normal(p[k].shape)
    return p


def _fields(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((nz, ny, nx)) * 3.0
    logk = rng.standard_normal((nz, ny, nx))
    e = rng.standard_normal((nz, ny, nx))
    return r, logk, e


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).reshape(-1)).cuda()


@pytest.mark.parametrize("shape", [(16, 8, 8), (32, 16, 24), (24, 40, 16)])
def test_forward_matches_oracle(rs, ctx, shape):
    import torch
    from oracle import convnet as cn
    p = _params(1)
    r, logk, _ = _fields(shape, 2)
    net = rs.Net(ctx, p, out_scale=5.0)
    out = torch.zeros(r.size, dtype=torch.float64, device="cuda")
    net.forward(shape, _dev(r), _dev(logk), out)
    got = out.cpu().numpy().reshape(r.shape)
    ref, _ = cn.forward(p, r, logk, out_scale=5.0, bf16=True)
    ref64, _ = cn.forward(p, r, logk, out_scale=5.0, bf16=False)
    assert rel(got, ref) <= 2e-2, rel(got, ref)
    assert rel(got, ref64) <= 5e-2


def test_forward_matches_oracle_with_tcgen05_on_two_levels(rs, ctx):
    """128 x 64 x 80: the second level (64 x 32 x 40) has 320 bricks of the
    tcgen05 kernel, two per SM and more, so its convolutions (e1a, e1b, and
    the decoder d1a with its upsampled input, d1b) run there too."""
    import torch
    from oracle import convnet as cn
    shape = (128, 64, 80)
    p = _params(3)
    r, logk, _ = _fields(shape, 4)
    net = rs.Net(ctx, p, out_scale=5.0)
    out = torch.zeros(r.size, dtype=torch.float64, device="cuda")
    net.forward(shape, _dev(r), _dev(logk), out)
    got = out.cpu().numpy().reshape(r.shape)
    ref, _ = cn.forward(p, r, logk, out_scale=5.0, bf16=True)
    assert rel(got, ref) <= 2e-2, rel(got, ref)


def test_gradients_match_oracle(rs, ctx):
    from oracle import convnet as cn
    shape = (16, 16, 8)
    p = _params(3)
    r, logk, e = _fields(shape, 4)
    e = e * 20.0
    net = rs.Net(ctx, p, out_scale=10.0)
    net.zero_grads()
    loss = net.accumulate(shape, _dev(r), _dev(logk), _dev(e), weight=1.0, want_loss=True)
    g = net.grads()
    out, cache = cn.forward(p, r, logk, out_scale=10.0, bf16=True)
    lref, gout = cn.loss_rel(out, e)
    gref = cn.backward(p, cache, gout, out_scale=10.0, bf16=True)
    assert abs(loss - lref) <= 2e-2 * lref
    for name in [k for k in p]:
        a, b = np.ravel(g[name]), np.ravel(gref[name])
        if np.linalg.norm(b) == 0:
            continue
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert rel(a, b) <= 6e-2 and cos >= 0.998, (name, rel(a, b), cos)


def test_training_reduces_loss_and_checkpoint_roundtrip(rs, ctx):
    shape = (16, 16, 16)
    p = _params(5)
    net = rs.Net(ctx, p, out_scale=1.0)
    rng = np.random.default_rng(6)
    logk = _dev(rng.standard_normal(shape[::-1]))
    r = _dev(rng.standard_normal(shape[::-1]))
    e = _dev(0.5 * rng.standard_normal(shape[::-1]))
    losses = []
    for _ in range(40):
        losses.append(net.accumulate(shape, r, logk, e, 1.0, want_loss=True))
        net.adam(lr=3e-3)
    assert losses[-1] < 0.7 * losses[0], losses[::8]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "net.bin")
        net.save(path)
        net2 = rs.Net(ctx, path=path)
        a, b = net.params(), net2.params()
        for k in a:
            assert np.array_equal(a[k], b[k])


def test_learned_cpr_fgmres_converges_and_falls_back(rs, ctx, orc):
    import torch
    g = synth.Grid(32, 32, 16)
    d = synth.pressure_7pt(g, 9)
    Ao = orc.Mat.csr(d)
    b = orc.spmv(Ao, synth.x_true(g.n, 9))
    A = rs.Mat.csr(ctx, d)
    for bad in (False, True):
        p = _params(7)
        if bad:
            p["head.b"] = np.array([np.nan])     # non-finite output: ILU(0) fallback
        net = rs.Net(ctx, p, out_scale=1.0)
        M = rs.Precond(ctx, A, "cpr_learned", net=net, log_perm=d["logk"], grid=(g.nx, g.ny, g.nz))
        x = rs.Vec.zeros(ctx, g.n)
        info = rs.solve_fgmres(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8)
        xs = x.numpy()
        assert info["status"] == 0, info
        assert orc.norm2(b - orc.spmv(Ao, xs)) / orc.norm2(b) <= 1e-8


def test_trained_checkpoint_gain_over_ilu0(rs, ctx, orc):
    """What the trained network adds: on a held-out field the learned
    two-stage preconditioner needs well under half the iterations of
    ILU(0) alone, and both reach the true residual."""
    path = os.path.join(os.path.dirname(rs.__file__), "models", "pressure_unet_64.bin")
    net = rs.Net(ctx, path=path)
    g = synth.Grid(64, 64, 64)
    d = synth.pressure_7pt(g, 2007)
    Ao = orc.Mat.csr(d)
    b = orc.spmv(Ao, synth.x_true(g.n, 2007))
    A = rs.Mat.csr(ctx, d)
    its = {}
    for name, M, fn in (("ilu0", rs.Precond(ctx, A, "ilu0"), rs.solve_gmres),
                        ("learned", rs.Precond(ctx, A, "cpr_learned", net=net, log_perm=d["logk"],
                                               grid=(g.nx, g.ny, g.nz)), rs.solve_fgmres)):
        x = rs.Vec.zeros(ctx, g.n)
        info = fn(A, M, rs.Vec(ctx, b), x, restart=30, rtol=1e-8)
        assert info["status"] == 0
        assert orc.norm2(b - orc.spmv(Ao, x.numpy())) / orc.norm2(b) <= 1e-8
        its[name] = info["iters"]
    assert its["learned"] <= 0.5 * its["ilu0"], its


def test_learned_cpr_graph_replays_match_the_direct_apply(rs, ctx):
    """From the second apply on, a CPR apply is replayed from a CUDA graph.
    Replays give the first (direct) apply's result bit for bit, also after a
    forward pass on another grid has reallocated the network's workspace,
    which the graph captured (the graph is then captured again)."""
    import torch
    g = synth.Grid(32, 32, 16)
    d = synth.pressure_7pt(g, 9)
    A = rs.Mat.csr(ctx, d)
    net = rs.Net(ctx, _params(7), out_scale=1.0)
    M = rs.Precond(ctx, A, "cpr_learned", net=net, log_perm=d["logk"], grid=(g.nx, g.ny, g.nz))
    r = rs.Vec(ctx, np.random.default_rng(3).standard_normal(g.n))
    outs = []
    for i in range(5):
        if i == 3:
            shape = (16, 8, 8)
            rr, lk, _ = _fields(shape, 1)
            out = torch.zeros(rr.size, dtype=torch.float64, device="cuda")
            net.forward(shape, _dev(rr), _dev(lk), out)
        z = rs.Vec.zeros(ctx, g.n) if i == 0 else z
        M.apply(r, z)
        outs.append(z.numpy().copy())
    assert np.isfinite(outs[0]).all()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
