"""Benchmark: time to a 1e-8 relative residual for preconditioned Krylov solves.

Default workload (one GPU): the 3-D 7-point pressure matrix on a 128x128x64
grid (1,048,576 cells, vertical permeability x0.1, log-normal permeability,
seed 1), b = A x_true, GMRES(30) right-preconditioned by ILU(0), all FP64,
rtol 1e-8, x0 = 0.  One step = one complete solve; the matrix, b and the
preconditioner are resident in HBM before the timed region (preconditioner
setup is timed separately).  Between timed steps a 512 MB buffer is written
to flush the 129 MB L2.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "time to 1e-8 rel. residual (s), learned vs ILU(0) precond; SpMV/ILU HBM GB/s"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "gmres_ilu0_128x128x64": dict(grid=(128, 128, 64), kz=0.1, solver="gmres", precond="ilu0",
                                  prec="fp64", restart=30),
    "gmres_ilu0_mixed_128x128x64": dict(grid=(128, 128, 64), kz=0.1, solver="gmres", precond="ilu0",
                                        prec="mixed", restart=30),
    "bicgstab_ilu0_128x128x64": dict(grid=(128, 128, 64), kz=0.1, solver="bicgstab", precond="ilu0",
                                     prec="fp64", restart=30),
    "gmres_ilu0_32x32x32": dict(grid=(32, 32, 32), kz=1.0, solver="gmres", precond="ilu0",
                                prec="fp64", restart=30),
}
DEFAULT = "gmres_ilu0_128x128x64"
RTOL = 1e-8
SEED = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rs", choices=["rs", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def build_problem(w):
    g = synth.Grid(*w["grid"])
    d = synth.pressure_7pt(g, SEED, kz_scale=w["kz"])
    xt = synth.x_true(g.n, SEED)
    return g, d, xt


# ----------------------------------------------------------------------------
# algorithmic bytes per launch (FP64 values 8 B, FP32 4 B, indices 4 B)
# ----------------------------------------------------------------------------
def algorithmic_bytes(d, prec):
    n = d["n"]
    nnz = d["col"].size
    nnz_l = (nnz - n) // 2
    vb = 4 if prec == "mixed" else 8
    return {
        # values + column indices + row pointers, x read once, y written once
        "spmv": 12 * nnz + 4 * (n + 1) + 16 * n,
        # strict-lower factor (value + index), r in, y out
        "l_sweep": (vb + 4) * nnz_l + 8 * n + vb * n,
        # strict-upper factor, reciprocal diagonal, y in, z out
        "u_sweep": (vb + 4) * nnz_l + vb * n + vb * n + 8 * n,
    }


def cgs_bytes(n, iters, m):
    """Total algorithmic bytes of the three CGS2 kernels over a solve with
    `iters` Arnoldi steps: step i reads the i+1 basis vectors once per pass."""
    tot = {"cgs_dots": 0, "cgs_update_dots": 0, "cgs_update_norm": 0}
    for it in range(iters):
        nc = it % m + 1
        tot["cgs_dots"] += 8 * n * (nc + 1)
        tot["cgs_update_dots"] += 8 * n * (nc + 2)
        tot["cgs_update_norm"] += 8 * n * (nc + 2)
    return tot


def source_sha(kernel):
    f = {"spmv": "rs_core.cu", "l_sweep": "rs_ilu.cu", "u_sweep": "rs_ilu.cu"}.get(kernel, "rs_krylov.cu")
    p = os.path.join(ROOT, "paper_1701_05913_gb300", "csrc", f)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(workload, {}).get(kernel)
        if e and e.get("source_sha") == source_sha(kernel):
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ----------------------------------------------------------------------------
def oracle_solve(w, d, xt, maxit=10000):
    """The CPU oracle's solve of the same system (single thread, FP64):
    returns (solve seconds, setup seconds, iterations)."""
    import oracle
    oracle.build()
    A = oracle.Mat.csr(d)
    b = oracle.spmv(A, xt)
    t0 = time.perf_counter()
    M = oracle.PC(A, w["precond"], mixed=(w["prec"] == "mixed"))
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    if w["solver"] == "bicgstab":
        _, info, _ = oracle.bicgstab(A, M, b, rtol=RTOL, maxit=maxit)
    else:
        _, info, _ = oracle.gmres(A, M, b, restart=w["restart"], rtol=RTOL, maxit=maxit)
    return time.perf_counter() - t0, setup, info["iters"]


def run_reference(args, w, rank, world):
    """The oracle as the reference arm: the first warm-up step is one full
    solve (its iteration count); every other step times one GMRES cycle (30
    iterations) of the same solve and scales it to that count."""
    if rank != 0:
        return
    g, d, xt = build_problem(w)
    full_s, setup, full_iters = oracle_solve(w, d, xt)
    sample = 30
    per = []
    for s in range(max(args.warmup - 1, 0) + args.steps):
        t, su, done = oracle_solve(w, d, xt, maxit=sample)
        if s >= args.warmup - 1:
            per.append(t / done * full_iters + su)
    v = statistics.median(per)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(w["grid"]), "n": g.n, "nnz": int(d["col"].size),
                   "solver": w["solver"], "precond": w["precond"], "precision": w["prec"], "rtol": RTOL},
        "iters": full_iters, "full_solve_s": full_s + setup,
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": "one full solve (%d iterations, %.2f s) then, per step, %d iterations of "
                                   "the same solve scaled to %d iterations plus ILU(0) setup"
                                   % (full_iters, full_s + setup, sample, full_iters)},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_gpu(args, w, rank, world, local):
    import torch

    import paper_1701_05913_gb300 as rs

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ctx = rs.Context(local)
    stream = torch.cuda.current_stream()
    g, d, xt = build_problem(w)
    A = rs.Mat.csr(ctx, d)
    xtv = rs.Vec(ctx, xt)
    b = rs.Vec.zeros(ctx, g.n)
    A.spmv(xtv, b)
    ctx.sync()
    t0 = time.perf_counter()
    M = rs.Precond(ctx, A, w["precond"], prec=w["prec"])
    ctx.sync()
    setup_s = time.perf_counter() - t0
    x = rs.Vec.zeros(ctx, g.n)

    def solve():
        if w["solver"] == "bicgstab":
            return rs.solve_bicgstab(A, M, b, x, rtol=RTOL)
        return rs.solve_gmres(A, M, b, x, restart=w["restart"], rtol=RTOL)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        x.t.zero_()
        info = solve()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # timed region: K complete solves, L2 flushed between them, profiler on
    clocks = ClockSampler(local)
    clocks.start()
    ctx.prof_enable(True)
    ctx.prof_read(reset=True)
    n_launch0 = ctx.launches()
    evs = []
    infos = []
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        x.t.zero_()
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(solve())
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    launches = ctx.launches() - n_launch0
    prof = ctx.prof_read(reset=True)
    ctx.prof_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b_) for a, b_ in evs]
    ms = sum(step_ms) / len(step_ms)

    # same solves without the profiler (its event records add host work)
    evs2 = []
    for _ in range(args.steps):
        x.t.zero_()
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solve()
        e1.record(stream)
        evs2.append((e0, e1))
    torch.cuda.synchronize()
    ms_noprof = sum(a.elapsed_time(b_) for a, b_ in evs2) / len(evs2)

    # end to end through the C ABI with host buffers: b from pinned host memory,
    # x back to pinned host memory, both copies inside the timed region
    hb = torch.from_numpy(b.numpy()).pin_memory()
    hx = torch.empty(g.n, dtype=torch.float64).pin_memory()
    L = rs.lib()
    e2e = []
    for _ in range(args.steps):
        x.t.zero_()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.rs_vec_set(b.h, rs._vp(hb.data_ptr()), rs.MEM_HOST)
        solve()
        L.rs_vec_get(x.h, rs._vp(hx.data_ptr()), rs.MEM_HOST)
        e2e.append(time.perf_counter() - t1)
    e2e_s = statistics.median(e2e)

    # max over ranks
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([ms, ms_noprof, e2e_s, wall], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms, ms_noprof, e2e_s, wall = tt.tolist()

    # roofline of the dominant kernel class, from the live profile
    peak, peak_src = measured_peaks()
    alg = algorithmic_bytes(d, w["prec"])
    iters = [i["iters"] for i in infos]
    cb = cgs_bytes(g.n, sum(iters), w["restart"])
    kern_ms = {k: v[0] for k, v in prof.items() if v[1] > 0}
    kern_n = {k: v[1] for k, v in prof.items() if v[1] > 0}
    dom = max(kern_ms, key=kern_ms.get)
    total_prof = sum(kern_ms.values())
    bytes_total = {k: alg[k] * kern_n[k] for k in ("spmv", "l_sweep", "u_sweep") if k in kern_n}
    bytes_total.update({k: cb[k] for k in cb if k in kern_n})
    achieved = {k: bytes_total[k] / (kern_ms[k] * 1e-3) / 1e9 for k in bytes_total}
    per_launch = bytes_total.get(dom, 0) / max(kern_n.get(dom, 1), 1)
    dom_ms = kern_ms[dom] / kern_n[dom]
    roofline = {
        "kernel": dom, "bound": "hbm", "achieved": round(achieved.get(dom, 0.0), 2), "peak": peak,
        "unit": "GB/s", "frac": round(achieved.get(dom, 0.0) / peak, 4),
        "traffic": ncu_traffic(dom, args.workload),
        "peak_source": peak_src, "alg_bytes_per_launch": int(per_launch), "avg_launch_us": round(dom_ms * 1e3, 2),
        "share_of_kernel_time": round(kern_ms[dom] / total_prof, 3),
    }

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        t, setup, done = oracle_solve(w, d, xt)
        cpu = {"value": t + setup, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": "one full solve of the same system on one host core (%d iterations; "
                         "ILU(0) setup %.3f s included)" % (done, setup)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if w["prec"] == "fp64" else "f64+f32", "data": "synthetic",
            "config": {"workload": args.workload, "grid": list(w["grid"]), "n": g.n, "nnz": int(d["col"].size),
                       "solver": "%s(%d)" % (w["solver"], w["restart"]) if w["solver"] == "gmres" else w["solver"],
                       "precond": w["precond"], "precision": w["prec"], "rtol": RTOL, "seed": SEED,
                       "l2": "flushed between steps (512 MB write)", "parallelism": "replicas" if world > 1 else "1 gpu"},
            "iters": statistics.median(iters),
            "true_rel_res": max(i["true_rel_res"] for i in infos),
            "setup_s": setup_s,
            "ms_per_step_without_profiler": ms_noprof,
            "wall_s": wall,
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * g.n, "d2h_bytes_per_step": 8 * g.n},
            "gpu_launches": launches,
            "roofline": roofline,
            "kernels": {k: {"ms_per_step": round(kern_ms[k] / args.steps, 4), "launches_per_step": kern_n[k] / args.steps,
                            "share": round(kern_ms[k] / total_prof, 4),
                            **({"GBs": round(achieved[k], 1)} if k in achieved else {})} for k in kern_ms},
            "spmv_GBs": round(achieved.get("spmv", 0.0), 1),
            "ilu_apply_GBs": round((bytes_total.get("l_sweep", 0) + bytes_total.get("u_sweep", 0)) /
                                   ((kern_ms.get("l_sweep", 1e-9) + kern_ms.get("u_sweep", 0)) * 1e-3) / 1e9, 1),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    run_gpu(args, w, rank, world, local)


if __name__ == "__main__":
    main()
