"""Pins of the learned-stage oracle (oracle/convnet.py), CPU only."""
import numpy as np
import pytest

from oracle import convnet as cn


def test_conv3_equals_im2col_product():
    rng = np.random.default_rng(0)
    D, H, W, ci, co = 3, 4, 5, 3, 2
    x = rng.standard_normal((D, H, W, ci))
    Wt = rng.standard_normal((3, 3, 3, co, ci))
    b = rng.standard_normal(co)
    # im2col built cell by cell: column (tap, ci), zero outside the grid
    cols = np.zeros((D * H * W, 27 * ci))
    row = 0
    for z in range(D):
        for y in range(H):
            for xx in range(W):
                t = 0
                for dz in range(3):
                    for dy in range(3):
                        for dx in range(3):
                            zz, yy, x2 = z + dz - 1, y + dy - 1, xx + dx - 1
                            if 0 <= zz < D and 0 <= yy < H and 0 <= x2 < W:
                                cols[row, t * ci:(t + 1) * ci] = x[zz, yy, x2]
                            t += 1
                row += 1
    Wmat = Wt.reshape(27, co, ci).transpose(0, 2, 1).reshape(27 * ci, co)
    ref = (cols @ Wmat + b).reshape(D, H, W, co)
    assert np.allclose(cn.conv3(x, Wt, b), ref, rtol=1e-13, atol=1e-13)


def test_conv3_delta_response_is_flipped_kernel():
    Wt = np.random.default_rng(1).standard_normal((3, 3, 3, 1, 1))
    x = np.zeros((5, 5, 5, 1))
    x[2, 2, 2, 0] = 1.0
    out = cn.conv3(x, Wt, np.zeros(1))[1:4, 1:4, 1:4, 0]
    assert np.allclose(out, Wt[::-1, ::-1, ::-1, 0, 0], rtol=0, atol=0)


def test_pool_upsample_adjoint():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((2, 3, 4, 5))
    b = rng.standard_normal((4, 6, 8, 5))
    # nearest upsampling is the adjoint of 2x2x2 sum pooling (= 8 x average)
    assert np.isclose(np.sum(cn.upsample2(a) * b), 8.0 * np.sum(a * cn.avgpool2(b)))
    assert np.allclose(cn.avgpool2_backward(cn.avgpool2(np.ones((4, 4, 4, 1)))), 1.0 / 8.0)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -3.14159, 1e-40, 65504.0])
    r = cn.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0                       # tie to even
    assert r[2] == 1.0 + 2.0 ** -7                          # rounds up
    assert abs(r[3] + 3.140625) < 1e-12
    assert cn.bf16_round(np.array([np.nan]))[0] != cn.bf16_round(np.array([np.nan]))[0]


def test_network_gradients_finite_difference():
    rng = np.random.default_rng(3)
    g = (8, 8, 8)
    p = cn.init_params(5)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    r = rng.standard_normal(g)
    logk = rng.standard_normal(g)
    e = rng.standard_normal(g)

    def L(pp, rr=r):
        out, _ = cn.forward(pp, rr, logk, out_scale=3.0)
        return cn.loss_rel(out, e)[0]

    out, cache = cn.forward(p, r, logk, out_scale=3.0)
    _, gout = cn.loss_rel(out, e)
    grads = cn.backward(p, cache, gout, out_scale=3.0)
    h = 1e-6
    for name in ["e0a.W", "e2b.W", "e3a.b", "d2a.W", "d1b.b", "d0a.W", "d0b.W", "head.W", "head.b"]:
        idx = tuple(rng.integers(0, s) for s in p[name].shape)
        pp = {k: v.copy() for k, v in p.items()}
        pp[name][idx] += h
        lp = L(pp)
        pp[name][idx] -= 2 * h
        lm = L(pp)
        fd = (lp - lm) / (2 * h)
        an = grads[name][idx]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, fd, an)
