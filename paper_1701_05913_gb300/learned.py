"""Training data, training loop and evaluation of the learned pressure stage.

Host-side driver only: every solve, SpMV, network pass and optimiser step
runs in librs.so through the C ABI.

Training pairs (r, e = A^{-1} r) come from the plain solver on seeded
permeability fields: for each field,
  * r = white noise and e from GMRES(30)+ILU(0) solved to a 1e-11 relative
    residual;
  * the residual and error after k GMRES(30)+ILU(0) iterations on
    b = A x_true (k = 5 and 20): r_k = b - A x_k, e_k = x_true - x_k
    (exact, since A e_k = r_k).
Loss: ||net(r) - e||^2 / ||e||^2 per pair, Adam, cosine learning-rate decay.
"""
from __future__ import annotations

import math
import time

import numpy as np

import synth

from . import Context, Mat, Net, Precond, Vec, solve_fgmres, solve_gmres, vec_axpbyz, vec_norm2  # noqa: F401


def _torch():
    import torch
    return torch


def make_pairs(ctx: Context, seeds, grid=(64, 64, 64), kz=1.0, noise_rtol=1e-11, ks=(5, 20)):
    """Returns a dict with device tensors: logk [F, n], r [P, n], e [P, n],
    field index of each pair [P], plus timing."""
    torch = _torch()
    g = synth.Grid(*grid)
    t0 = time.perf_counter()
    logks, rs_, es, fidx = [], [], [], []
    for fi, s in enumerate(seeds):
        d = synth.pressure_7pt(g, s, kz_scale=kz)
        A = Mat.csr(ctx, d)
        M = Precond(ctx, A, "ilu0")
        logks.append(torch.from_numpy(d["logk"]).cuda())
        rng = np.random.default_rng(10_000 + s)
        # white-noise right-hand side, solved accurately
        r = Vec(ctx, rng.standard_normal(g.n))
        e = Vec.zeros(ctx, g.n)
        solve_gmres(A, M, r, e, restart=30, rtol=noise_rtol, maxit=20000)
        rs_.append(r.t.clone())
        es.append(e.t.clone())
        fidx.append(fi)
        # Krylov residuals and errors of a plain solve
        xt = Vec(ctx, synth.x_true(g.n, s))
        b = Vec.zeros(ctx, g.n)
        A.spmv(xt, b)
        for k in ks:
            x = Vec.zeros(ctx, g.n)
            solve_gmres(A, M, b, x, restart=30, rtol=1e-14, maxit=k)
            rk = Vec(ctx, b.t.clone())
            A.amxpby(-1.0, x, 1.0, rk)          # r_k = b - A x_k
            ek = Vec.zeros(ctx, g.n)
            vec_axpbyz(1.0, xt, -1.0, x, ek)    # e_k = x_true - x_k
            rs_.append(rk.t.clone())
            es.append(ek.t.clone())
            fidx.append(fi)
    ctx.sync()
    return dict(grid=grid, logk=torch.stack(logks), r=torch.stack(rs_), e=torch.stack(es),
                field=torch.tensor(fidx), seconds=time.perf_counter() - t0)


def output_scale(ctx: Context, data) -> float:
    """Median over the pairs of rms(e) / rms(r) = ||e|| / ||r|| (fixes the
    network's output scale); the norms are the library's."""
    ratios = [vec_norm2(Vec(ctx, data["e"][i])) / vec_norm2(Vec(ctx, data["r"][i]))
              for i in range(data["r"].shape[0])]
    return float(np.median(ratios))


def he_params(seed: int = 0) -> dict:
    """He-normal initial weights (zero biases), drawn on the host."""
    rng = np.random.default_rng(seed)
    from . import NET_LAYERS
    p = {}
    for name, cin in NET_LAYERS:
        p[name + ".W"] = rng.standard_normal((3, 3, 3, 16, cin)) * math.sqrt(2.0 / (27 * cin))
        p[name + ".b"] = np.zeros(16)
    p["head.W"] = rng.standard_normal((1, 16)) * math.sqrt(1.0 / 16)
    p["head.b"] = np.zeros(1)
    return p


def train_net(ctx: Context, data, epochs=8, batch=8, lr=2e-3, seed=0, net: Net | None = None, log=None):
    """Adam on the relative-L2 loss with a cosine-decayed learning rate."""
    torch = _torch()
    grid = data["grid"]
    P = data["r"].shape[0]
    if net is None:
        net = Net(ctx, he_params(seed), out_scale=output_scale(ctx, data))
    rng = np.random.default_rng(seed)
    steps = epochs * max(P // batch, 1)
    hist = []
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = rng.permutation(P)
        ep_loss = 0.0
        for b0 in range(0, P - batch + 1, batch):
            idx = order[b0:b0 + batch]
            loss = 0.0
            for i in idx:
                f = int(data["field"][i])
                loss += net.accumulate(grid, data["r"][i], data["logk"][f], data["e"][i], 1.0 / batch,
                                       want_loss=True)
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / steps))
            net.adam(lr=lr_t)
            step += 1
            ep_loss += loss / batch
        nb = max(P // batch, 1)
        hist.append(ep_loss / nb)
        if log:
            log("epoch %d loss %.4f (%.1f s)" % (ep, ep_loss / nb, time.perf_counter() - t0))
    torch.cuda.synchronize()
    return net, dict(loss=hist, seconds=time.perf_counter() - t0, steps=step)


def evaluate(ctx: Context, net: Net, seeds, grid=(64, 64, 64), kz=1.0, rtol=1e-8, prec="fp64", repeats=1):
    """Held-out comparison on each seed: FGMRES(30) with the learned CPR stage
    vs GMRES(30)+ILU(0), both from x0 = 0 to rtol on b = A x_true.  Times
    are solve-only, in seconds, from CUDA events."""
    torch = _torch()
    g = synth.Grid(*grid)
    rows = []
    for s in seeds:
        d = synth.pressure_7pt(g, s, kz_scale=kz)
        A = Mat.csr(ctx, d)
        xt = Vec(ctx, synth.x_true(g.n, s))
        b = Vec.zeros(ctx, g.n)
        A.spmv(xt, b)
        Mi = Precond(ctx, A, "ilu0", prec=prec)
        Ml = Precond(ctx, A, "cpr_learned", prec=prec, net=net, log_perm=d["logk"], grid=grid)
        res = {}
        for name, fn, M in (("ilu0_gmres", solve_gmres, Mi), ("learned_fgmres", solve_fgmres, Ml)):
            best = None
            for _ in range(repeats + 1):
                x = Vec.zeros(ctx, g.n)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                info = fn(A, M, b, x, restart=30, rtol=rtol)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1e3
                best = t if best is None else min(best, t)
            dx = Vec.zeros(ctx, g.n)
            vec_axpbyz(1.0, x, -1.0, xt, dx)
            err = vec_norm2(dx) / vec_norm2(xt)
            res[name] = dict(iters=info["iters"], seconds=best, true_rel_res=info["true_rel_res"],
                             status=info["status"], err_vs_xtrue=err)
        rows.append(dict(seed=s, **res))
    return rows


def main(argv=None):
    """python -m paper_1701_05913_gb300.learned --out model.bin [--grid 64x64x64]
    [--train-seeds 1000:1200] [--eval-seeds 2000:2020] [--epochs 30]

    Generates the training pairs with the plain solver, trains the network,
    saves the checkpoint and prints one JSON line with the training history and
    the held-out comparison."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--grid", default="64x64x64")
    ap.add_argument("--train-seeds", default="1000:1200")
    ap.add_argument("--eval-seeds", default="2000:2020")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    grid = tuple(int(v) for v in a.grid.split("x"))
    t0, t1 = (int(v) for v in a.train_seeds.split(":"))
    e0, e1 = (int(v) for v in a.eval_seeds.split(":"))
    ctx = Context(0)
    data = make_pairs(ctx, list(range(t0, t1)), grid=grid)
    net, hist = train_net(ctx, data, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed,
                          log=lambda m: print(m, flush=True))
    net.save(a.out)
    rows = evaluate(ctx, net, list(range(e0, e1)), grid=grid)
    li = [r["learned_fgmres"]["iters"] for r in rows]
    bi = [r["ilu0_gmres"]["iters"] for r in rows]
    lt = [r["learned_fgmres"]["seconds"] for r in rows]
    bt = [r["ilu0_gmres"]["seconds"] for r in rows]
    print(json.dumps(dict(grid=grid, train_fields=t1 - t0, pairs=int(data["r"].shape[0]),
                          datagen_s=data["seconds"], train=hist, out_scale=output_scale(ctx, data),
                          eval=dict(seeds=[e0, e1], learned_iters_median=float(np.median(li)),
                                    ilu0_iters_median=float(np.median(bi)),
                                    learned_s_median=float(np.median(lt)), ilu0_s_median=float(np.median(bt)),
                                    max_true_rel_res=max(r["learned_fgmres"]["true_rel_res"] for r in rows),
                                    rows=rows))), flush=True)


if __name__ == "__main__":
    main()
