"""CPU oracle of the learned pressure stage — TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this follows the network fixed for the
pressure stage of the two-stage CPR preconditioner: a 3-D U-Net over an
nz x ny x nx grid with four resolution levels, 16 channels, 3x3x3
convolutions with zero padding, ReLU, 2x2x2 average pooling down, nearest
x2 upsampling with skip concatenation, and a 1x1x1 output head.  Input
channels: the residual divided by its RMS, and the log-permeability.  The
output, times the residual's RMS and a fixed output scale, approximates
A^{-1} r.

Plain numpy in FP64: every convolution is a loop over the 27 taps with one
channel contraction per tap; backward passes are the explicit adjoints.  With
bf16=True the activations are rounded to bfloat16 (round to nearest even)
where the CUDA path stores bfloat16, and weights are rounded likewise.

Tensors are (z, y, x, c) arrays; conv weights are (3, 3, 3, cout, cin)
indexed [dz, dy, dx, co, ci] with tap offset (dz-1, dy-1, dx-1).

Parity status: pinned by tests/test_convnet_pins.py (im2col product, delta
response, adjointness, finite-difference gradients).
"""
from __future__ import annotations

import numpy as np

CH = 16
LEVELS = 4

# layer names in order, with (cin, cout)
LAYERS = [
    ("e0a", 2, CH), ("e0b", CH, CH),
    ("e1a", CH, CH), ("e1b", CH, CH),
    ("e2a", CH, CH), ("e2b", CH, CH),
    ("e3a", CH, CH), ("e3b", CH, CH),
    ("d2a", 2 * CH, CH), ("d2b", CH, CH),
    ("d1a", 2 * CH, CH), ("d1b", CH, CH),
    ("d0a", 2 * CH, CH), ("d0b", CH, CH),
]


def bf16_round(x):
    """Round float64 values to bfloat16 (via float32, round to nearest even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = r.astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out.astype(np.float64)


def conv3(x, W, b):
    """out[z,y,x,o] = b[o] + sum_{taps, ci} W[dz,dy,dx,o,ci] x[z+dz-1, y+dy-1, x+dx-1, ci]."""
    D, H, Wd, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((D, H, Wd, W.shape[3])) + b
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += np.einsum("zyxc,oc->zyxo", xp[dz:dz + D, dy:dy + H, dx:dx + Wd], W[dz, dy, dx])
    return out


def conv3_backward(x, W, g):
    """Gradients of conv3 given g = dL/dout: (dx, dW, db)."""
    D, H, Wd, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = (slice(dz, dz + D), slice(dy, dy + H), slice(dx, dx + Wd))
                dW[dz, dy, dx] = np.einsum("zyxo,zyxc->oc", g, xp[sl])
                dxp[sl] += np.einsum("zyxo,oc->zyxc", g, W[dz, dy, dx])
    return dxp[1:-1, 1:-1, 1:-1], dW, g.sum(axis=(0, 1, 2))


def avgpool2(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def avgpool2_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def upsample2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def upsample2_backward(g):
    D, H, W, C = g.shape
    return g.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def init_params(seed: int = 0):
    """He-normal weights from numpy's generator (the CUDA path receives these
    arrays; it does not draw its own)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, cin, cout in LAYERS:
        p[name + ".W"] = rng.standard_normal((3, 3, 3, cout, cin)) * np.sqrt(2.0 / (27 * cin))
        p[name + ".b"] = np.zeros(cout)
    p["head.W"] = rng.standard_normal((1, CH)) * np.sqrt(1.0 / CH)
    p["head.b"] = np.zeros(1)
    return p


def forward(p, r, logk, out_scale=1.0, bf16=False):
    """Network output e_hat (z, y, x) for residual r and log-permeability logk
    (both (z, y, x)); returns (e_hat, cache)."""
    q = (lambda a: bf16_round(a)) if bf16 else (lambda a: a)
    rms = np.sqrt(np.mean(r * r))
    rms = rms if rms > 0 else 1.0
    x = q(np.stack([r / rms, logk], axis=-1))
    cache = {"in": x, "rms": rms}
    W = {k: (q(v) if k.endswith(".W") else v) for k, v in p.items()}

    def cr(name, inp):
        pre = conv3(inp, W[name + ".W"], W[name + ".b"])
        out = q(np.maximum(pre, 0.0))
        cache[name] = (inp, pre, out)
        return out

    s = []
    h = x
    for lvl in range(LEVELS):
        if lvl > 0:
            h = q(avgpool2(h))
        h = cr("e%da" % lvl, h)
        h = cr("e%db" % lvl, h)
        s.append(h)
    for lvl in range(LEVELS - 2, -1, -1):
        up = upsample2(h)
        h = cr("d%da" % lvl, np.concatenate([up, s[lvl]], axis=-1))
        h = cr("d%db" % lvl, h)
    cache["last"] = h
    e = h @ W["head.W"][0] + W["head.b"][0]
    return e * rms * out_scale, cache


def backward(p, cache, g_out, out_scale=1.0, bf16=False):
    """Gradients of a scalar loss w.r.t. every parameter (and the input
    channels, key "input"), given g_out = dL/de_hat.  Rounding to bfloat16 in
    the forward pass is treated as the identity."""
    q = (lambda a: bf16_round(a)) if bf16 else (lambda a: a)
    W = {k: (q(v) if k.endswith(".W") else v) for k, v in p.items()}
    grads = {}
    ge = g_out * cache["rms"] * out_scale
    h = cache["last"]
    grads["head.W"] = np.einsum("zyx,zyxc->c", ge, h)[None, :]
    grads["head.b"] = np.array([ge.sum()])
    return _backward_ordered(p, cache, ge, W, grads)


def _backward_ordered(p, cache, ge, W, grads):
    def cr_back(name, g):
        inp, pre, out = cache[name]
        gp = g * (pre > 0)
        gi, dW, db = conv3_backward(inp, W[name + ".W"], gp)
        grads[name + ".W"] = dW
        grads[name + ".b"] = db
        return gi

    gh = ge[..., None] * W["head.W"][0]
    gskip = [np.zeros(0)] * LEVELS
    # decoder, fine to coarse: d0 -> d1 -> d2, each passing its gradient to
    # the upsampled coarser output and to its skip input
    for lvl in range(0, LEVELS - 1):
        gh = cr_back("d%db" % lvl, gh)
        gi = cr_back("d%da" % lvl, gh)
        gskip[lvl] = gi[..., CH:]
        gh = upsample2_backward(gi[..., :CH])
    # encoder, coarse to fine
    for lvl in range(LEVELS - 1, -1, -1):
        if lvl < LEVELS - 1:
            gh = gh + gskip[lvl]
        gh = cr_back("e%db" % lvl, gh)
        gh = cr_back("e%da" % lvl, gh)
        if lvl > 0:
            gh = avgpool2_backward(gh)
    grads["input"] = gh
    return grads


def loss_rel(e_hat, e):
    """Relative squared error ||e_hat - e||^2 / ||e||^2 and its gradient."""
    d = e_hat - e
    den = np.sum(e * e)
    return np.sum(d * d) / den, 2.0 * d / den
