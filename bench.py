"""Benchmark: time to a 1e-8 relative residual for preconditioned Krylov solves.

Default workload (one GPU): the largest configuration of the metric, the
black-oil-like 3x3-block system on a 128^3 grid (2,097,152 cells, 6,291,456
unknowns, seed 1), b = A x_true, FGMRES(30) right-preconditioned by the
two-stage CPR whose pressure stage is the learned U-Net (BF16), block ILU(0)
second stage with FP32 factors, FP64 outer iteration, rtol 1e-8, x0 = 0.
The same line times the same solve with the ILU(0) pressure stage
(`baseline_method`).  One step = one complete solve; matrices, right-hand
sides and preconditioners are resident in HBM before the timed region
(setup is timed separately).  A 512 MB buffer is written between timed
steps to flush the 129 MB L2.

Other workloads (--workload): the 32^3 and 128x128x64 scalar systems with
GMRES(30)/BiCGSTAB/CG + ILU(0), FP64 or mixed; the learned pressure stage on
64^3 held-out fields (FGMRES(30), learned two-stage CPR vs
GMRES(30)+ILU(0)); the 100x100x50 black-oil-like 3x3-block system with
CPR-FGMRES(30); RAS, AMG and LGMRES variants.

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
# the CPU oracle is timed on one host core: numpy's BLAS (the oracle
# network's channel contractions) must not start threads of its own
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "time to 1e-8 rel. residual (s), learned vs ILU(0) precond; SpMV/ILU HBM GB/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
RTOL = 1e-8
NET_PATH = os.path.join(ROOT, "paper_1701_05913_gb300", "models", "pressure_unet_64.bin")

WORKLOADS = {
    "gmres_ilu0_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="gmres", precond="ilu0",
                                  prec="fp64"),
    "gmres_ilu0_mixed_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="gmres",
                                        precond="ilu0", prec="mixed"),
    "bicgstab_ilu0_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="bicgstab",
                                     precond="ilu0", prec="fp64"),
    "gmres_ilu0_32x32x32": dict(kind="csr", grid=(32, 32, 32), kz=1.0, solver="gmres", precond="ilu0",
                                prec="fp64"),
    "learned_fgmres_64x64x64": dict(kind="learned", grid=(64, 64, 64), kz=1.0, solver="fgmres",
                                    precond="cpr_learned", prec="fp64", seeds=list(range(2000, 2020))),
    "cpr_fgmres_bsr3_100x100x50": dict(kind="bsr", grid=(100, 100, 50), kz=1.0, solver="fgmres",
                                       precond="cpr", prec="fp64"),
    "cpr_fgmres_bsr3_mixed_100x100x50": dict(kind="bsr", grid=(100, 100, 50), kz=1.0, solver="fgmres",
                                             precond="cpr", prec="mixed"),
    "cpr_learned_bsr3_128x128x128": dict(kind="bsr_learned", grid=(128, 128, 128), kz=1.0, solver="fgmres",
                                         precond="cpr_learned", prec="mixed"),
    "cg_ilu0_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="cg", precond="ilu0",
                               prec="fp64"),
    # LGMRES (the aug_k setting of Sec. 3): GMRES(30) cycles augmented with the last 3 corrections
    "lgmres_ilu0_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="lgmres", precond="ilu0",
                                   prec="fp64", aug_k=3),
    # algebraic multigrid (Sec. 4.2, Algs. 3-4): PCG with one V-cycle per iteration
    "cg_amg_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="cg", precond="amg", prec="fp64",
                              amg=dict()),
    # the same with Fig. 34's hybrid Gauss-Seidel relaxation (32-row chunks)
    "cg_amg_hgs_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="cg", precond="amg",
                                  prec="fp64", amg=dict(smoother=1)),
    # the paper's CPR with an AMG pressure stage (Sec. 4.2.1, Alg. 6 with M_p = one V-cycle)
    "cpr_amg_fgmres_bsr3_100x100x50": dict(kind="bsr", grid=(100, 100, 50), kz=1.0, solver="fgmres",
                                           precond="cpr", prec="mixed", pstage="amg", amg=dict()),
    # the paper's production preconditioner (Example 4): BiCGSTAB + CPR-FPF (Alg. 7) whose F stage
    # is RAS with one layer of overlap (4 x 4 x 2 block subdomains) and whose P stage is AMG
    "cpr_fpf_ras_amg_bicgstab_bsr3_100x100x50": dict(kind="bsr", grid=(100, 100, 50), kz=1.0,
                                                     solver="bicgstab", precond="cpr", prec="mixed", form="fpf",
                                                     pstage="amg", amg=dict(),
                                                     ras=dict(parts=(4, 4, 2), overlap=1, level=0)),
    # restricted additive Schwarz (Sec. 4.1) with the paper's defaults (Fig. 31): one layer of
    # overlap, ILU(1) local solver; 8 x 8 x 4 boxes of 16^3 cells
    "gmres_ras_ilu1_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="gmres", precond="ras",
                                      prec="fp64", ras=dict(parts=(8, 8, 4), overlap=1, level=1)),
    # the same boxes with ILUT(p, tol) local solvers at Fig. 31's defaults (p = -1, tol = 1e-3)
    "gmres_ras_ilut_128x128x64": dict(kind="csr", grid=(128, 128, 64), kz=0.1, solver="gmres", precond="ras",
                                      prec="fp64", ras=dict(parts=(8, 8, 4), overlap=1, level=0, ilut=(-1, 1e-3))),
    # the paper's production pairing (Examples 2 and 4): BiCGSTAB + CPR-FPF (Alg. 7)
    "cpr_fpf_bicgstab_bsr3_100x100x50": dict(kind="bsr", grid=(100, 100, 50), kz=1.0, solver="bicgstab",
                                             precond="cpr", prec="mixed", form="fpf"),
}
DEFAULT = "cpr_learned_bsr3_128x128x128"
SEED = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rs", choices=["rs", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", default=None,
                    help="NX,NY,NZ: the workload's method on another grid (small cases for ncu captures; "
                         "the config then names the grid after the workload)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, bf16, src = FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, "fallback"
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            hbm = float(d.get("hbm_gbs", hbm))
            bf16 = float(d.get("bf16_tflops", bf16))
            src = "measured"
        except Exception:
            pass
    return hbm, bf16, src


# ----------------------------------------------------------------------------
# problems (host arrays from the seeded generators)
# ----------------------------------------------------------------------------
def host_problem(w, seed):
    g = synth.Grid(*w["grid"])
    if w["kind"] in ("bsr", "bsr_learned"):
        m = synth.black_oil_bsr3(g, seed, kz_scale=w["kz"])
        xt = synth.x_true(3 * g.n, seed)
        return g, m, xt
    d = synth.pressure_7pt(g, seed, kz_scale=w["kz"])
    return g, d, synth.x_true(g.n, seed)


# ----------------------------------------------------------------------------
# algorithmic bytes (FP64 8 B, FP32 4 B, int32 4 B) and FLOPs per launch
# ----------------------------------------------------------------------------
def scalar_ilu_bytes(n, nnz, vb):
    nnz_l = (nnz - n) // 2
    return {"l_sweep": (vb + 4) * nnz_l + 8 * n + vb * n,          # factor, r in, y out
            "u_sweep": (vb + 4) * nnz_l + vb * n + vb * n + 8 * n}   # factor, 1/u_ii, y in, z out


def block_ilu_bytes(nb, nnzb, vb):
    nl = (nnzb - nb) // 2
    return {"bl_sweep": (4 + 9 * vb) * nl + 24 * nb + 3 * vb * nb,
            "bu_sweep": (4 + 9 * vb) * nl + 9 * vb * nb + 3 * vb * nb + 24 * nb}


def net_flops(grid):
    nx, ny, nz = grid
    f = 0
    cins = [2, 16, 16, 16, 16, 16, 16, 16, 32, 16, 32, 16, 32, 16]
    lvls = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
    for cin, l in zip(cins, lvls):
        f += 2 * 27 * cin * 16 * (nx >> l) * (ny >> l) * (nz >> l)
    return f + 2 * 16 * nx * ny * nz


def kernel_model(w, A_host, ras_sizes=None):
    """Algorithmic bytes per launch of each kernel class.  For RAS the sweeps
    run over the stacked extended subdomains (ras_sizes = rows, entries)."""
    vb = 4 if w["prec"] == "mixed" else 8
    if w["kind"] in ("bsr", "bsr_learned"):
        nb, nnzb = A_host["nb"], A_host["bcol"].size
        # the CPR residual after the pressure stage (PF form) reads only the
        # pressure column of each block: 28 B a block, p, f and t
        mod = {"spmv": 76 * nnzb + 4 * (nb + 1) + 48 * nb,
               "cpr_resid": 28 * nnzb + 4 * (nb + 1) + 8 * nb + 48 * nb}
        mod.update(scalar_ilu_bytes(nb, nnzb, vb))
        mod.update(block_ilu_bytes(*(ras_sizes or (nb, nnzb)), vb))
        return mod, 3 * nb
    n, nnz = A_host["n"], A_host["col"].size
    mod = {"spmv": 12 * nnz + 4 * (n + 1) + 16 * n}
    mod.update(scalar_ilu_bytes(*(ras_sizes or (n, nnz)), vb))
    return mod, n


def box_partition(grid, parts):
    """Subdomain of every cell (x fastest) for px x py x pz boxes of the grid."""
    (nx, ny, nz), (px, py, pz) = grid, parts
    bx, by, bz = np.arange(nx) * px // nx, np.arange(ny) * py // ny, np.arange(nz) * pz // nz
    return ((bz[:, None, None] * py + by[None, :, None]) * px + bx[None, None, :]).reshape(-1).astype(np.int32)


def ras_kwargs(w):
    """Precond arguments of a RAS workload: box subdomains of the grid."""
    r = w["ras"]
    return dict(nparts=int(np.prod(r["parts"])), part=box_partition(w["grid"], r["parts"]),
                overlap=r["overlap"], level=r["level"], **({"ilut": r["ilut"]} if "ilut" in r else {}))


def amg_vcycle_model(w, sizes):
    """SpMV launches and algorithmic bytes of one V-cycle: on every level
    above the coarsest, 2 nu residuals with A_l (one with hybrid
    Gauss-Seidel smoothing), one restriction, one
    prolongation (bytes of an r x c operator with z entries: 12 z + 4 (r+1)
    + 8 r + 8 c)."""
    nu = w.get("amg", {}).get("nu", 2)
    # with hybrid Gauss-Seidel the sweeps are their own kernel, not of the
    # SpMV class: only the residual remains there
    nres = 1 if w.get("amg", {}).get("smoother", 0) == 1 else 2 * nu
    launches, nbytes = 0, 0
    for l in range(len(sizes) - 1):
        n, za, zp = sizes[l]
        nc = sizes[l + 1][0]
        launches += nres + 2
        nbytes += nres * (12 * za + 4 * (n + 1) + 16 * n)
        nbytes += (12 * zp + 4 * (nc + 1) + 8 * nc + 8 * n) + (12 * zp + 4 * (n + 1) + 8 * n + 8 * nc)
    return {"launches": launches, "bytes": nbytes}


def executed_launches(w, infos, amg_vc=None, spmv_bytes=None):
    """Launches that did work (the rest returned at once on the device's
    cycle-done flag), per kernel class, from each solve's iteration and
    cycle counts.  GMRES: one SpMV and one preconditioner apply per Arnoldi
    step, one true-residual SpMV per cycle plus the final check, and (right
    preconditioning) one more apply per cycle for the update.  BiCGSTAB: two
    SpMVs and two applies per iteration."""
    cpr = w["precond"] in ("cpr", "cpr_learned")
    block = w["kind"] in ("bsr", "bsr_learned")
    cnt = {k: 0 for k in ("spmv", "l_sweep", "u_sweep", "bl_sweep", "bu_sweep", "net", "cpr_resid")}
    for info in infos:
        I, C = info["iters"], info["restarts"]
        if w["solver"] == "bicgstab":
            applies, spmv = 2 * I, 2 * I + 1
        elif w["solver"] == "cg":
            applies, spmv = I, I + C + 1
        elif w["solver"] == "lgmres":
            # cycle c (from 0) ends with min(c, aug_k) augmented steps, which
            # take an SpMV but no preconditioner apply (the last, converging
            # cycle is counted as if complete)
            aug = sum(min(c, w["aug_k"]) for c in range(C + 1))
            applies, spmv = max(I - aug, C + 1), I + C + 1
        else:
            applies = I + (0 if w["solver"] == "fgmres" else C)
            spmv = I + C + 1
        # CPR forms (Algs. 5-8): one residual between consecutive stages,
        # nF block-ILU(0) stages and nP pressure stages per apply
        form = w.get("form", "pf").upper() if cpr else "F"
        nF, nP = form.count("F"), form.count("P")
        if cpr:
            spmv += applies * (len(form) - 1)
            if block and form == "PF":
                # that residual takes the pressure-column kernel instead
                spmv -= applies
                cnt["cpr_resid"] += applies
        cnt["spmv"] += spmv
        if amg_vc:
            # every AMG V-cycle (the preconditioner, or CPR's pressure stage)
            # adds its SpMVs on all levels to the SpMV class
            vcs = applies * (nP if cpr else 1)
            cnt["spmv"] += vcs * amg_vc["launches"]
            cnt["_spmv_bytes"] = cnt.get("_spmv_bytes", 0) + spmv * spmv_bytes + vcs * amg_vc["bytes"]
        if w["precond"] == "cpr_learned":
            cnt["net"] += applies * nP
        if block:
            cnt["bl_sweep"] += applies * nF
            cnt["bu_sweep"] += applies * nF
            if w["precond"] == "cpr":
                cnt["l_sweep"] += applies * nP   # ILU(0) of the decoupled pressure matrix
                cnt["u_sweep"] += applies * nP
        else:
            cnt["l_sweep"] += applies * nF       # ILU(0) (or the CPR second stage on A)
            cnt["u_sweep"] += applies * nF
    return cnt


def cgs_bytes(n, iters_list, m=30):
    tot = {"cgs_dots": 0, "cgs_update_dots": 0, "cgs_update_norm": 0}
    for iters in iters_list:
        for it in range(iters):
            nc = it % m + 1
            tot["cgs_dots"] += 8 * n * (nc + 1)
            tot["cgs_update_dots"] += 8 * n * (nc + 2)
            tot["cgs_update_norm"] += 8 * n * (nc + 2)
    return tot


# The CGS2 passes are bound by the FP64 pipe: their useful multiply-adds per
# second against the GB300's nominal FP64 rate, 1.25 TFLOP/s = 625 G FMA/s (a
# DFMA throughput loop on this GPU measures 600 G/s)
FP64_FMA_PEAK = 625e9


def cgs_fmas(n, iters_list, m=30):
    """Useful FP64 multiply-adds of the three CGS2 passes: pass 1 h = V^T w
    and ||w||^2, pass 2 w -= V h and h' = V^T w, pass 3 w -= V h' and
    ||w||^2, for nc = i + 1 basis vectors at Arnoldi step i."""
    tot = {"cgs_dots": 0, "cgs_update_dots": 0, "cgs_update_norm": 0}
    for iters in iters_list:
        for it in range(iters):
            nc = it % m + 1
            tot["cgs_dots"] += n * (nc + 1)
            tot["cgs_update_dots"] += n * 2 * nc
            tot["cgs_update_norm"] += n * (nc + 1)
    return tot


def source_sha(kernel):
    files = {"spmv": ["rs_core.cu"], "net": ["rs_net.cu"], "cpr_resid": ["rs_precond.cu"]}.get(
        kernel, ["rs_ilu.cu", "rs_wave.cu"] if "sweep" in kernel else ["rs_krylov.cu"])
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1701_05913_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        e = json.load(open(p)).get(workload, {}).get(kernel)
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
        self.idx, self.proc, self.path = gpu_index, None, None

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
def _oracle_net_stage(net_params, out_scale, grid, logk, slab=None, clock=None):
    """The numpy network as the oracle's pressure stage.  With slab = k the
    network runs on the first k z-planes only (the rest of the correction is
    zero), so that a timing sample stays bounded: the network is fully
    convolutional and its cost is proportional to the voxels it covers.
    clock (a one-element list) accumulates the seconds spent in the network."""
    from oracle import convnet as cn
    nx, ny, nz = grid
    # the U-Net pools three times: a slab holds a multiple of 8 planes
    zs = nz if slab is None else max(8, min(int(slab) // 8 * 8, nz))

    def stage(rp):
        t0 = time.perf_counter()
        r3, k3 = rp.reshape(nz, ny, nx), logk.reshape(nz, ny, nx)
        out = np.zeros_like(r3)
        out[:zs], _ = cn.forward(net_params, r3[:zs], k3[:zs], out_scale=out_scale, bf16=True)
        if clock is not None:
            clock[0] += time.perf_counter() - t0
        return out.reshape(-1)
    return stage


def oracle_setup(w, A_host, xt, net_file=NET_PATH, net_slab=None):
    """The oracle's system, right-hand side and preconditioner for the
    workload.  With the learned stage the network runs on net_slab z-planes
    (all if None); the volume factor nz / net_slab scales its time to the
    full grid."""
    import oracle
    oracle.build()
    if w["kind"] in ("bsr", "bsr_learned"):
        A = oracle.Mat.bsr(A_host)
    else:
        A = oracle.Mat.csr(A_host)
    b = oracle.spmv(A, xt)
    mixed = w["prec"] == "mixed"
    clock, vol = [0.0], 1.0
    t0 = time.perf_counter()
    if w["precond"] == "cpr_learned":
        params, scale = load_net_host(net_file)
        nz = w["grid"][2]
        if net_slab is not None:
            vol = nz / max(8, min(int(net_slab) // 8 * 8, nz))
        M = oracle.PC(A, "cpr", mixed=mixed,
                      pstage=_oracle_net_stage(params, scale, w["grid"], A_host["logk"], net_slab, clock))
    elif w["precond"] == "amg":
        M = oracle.PC(A, "amg", amg=w["amg"])
    elif w.get("pstage") == "amg":
        kr = {}
        if "ras" in w:
            k = ras_kwargs(w)
            kr = dict(ras=dict(nsub=k["nparts"], part=k["part"], overlap=k["overlap"], level=k["level"]))
        M = oracle.PC(A, "cpr", mixed=mixed, form=w.get("form", "pf"), amg=w["amg"], **kr)
    elif w["precond"] == "ras":
        k = ras_kwargs(w)
        M = oracle.PC(A, "ras", ras=dict(nsub=k["nparts"], part=k["part"], overlap=k["overlap"], level=k["level"],
                                         **({"ilut": k["ilut"]} if "ilut" in k else {})))
    else:
        M = oracle.PC(A, w["precond"], mixed=mixed, form=w.get("form", "pf"))
    return dict(A=A, M=M, b=b, setup=time.perf_counter() - t0, clock=clock, vol=vol)


def oracle_solve(o, w, maxit):
    """One oracle solve from x0 = 0, at most maxit iterations: (seconds,
    iterations, seconds of it spent in the network)."""
    import oracle
    A, M, b = o["A"], o["M"], o["b"]
    o["clock"][0] = 0.0
    t0 = time.perf_counter()
    if w["solver"] == "lgmres":
        _, info = oracle.lgmres(A, M, b, restart=30, aug_k=w["aug_k"], rtol=RTOL, maxit=maxit)
    elif w["solver"] == "bicgstab":
        _, info, _ = oracle.bicgstab(A, M, b, rtol=RTOL, maxit=maxit)
    elif w["solver"] == "cg":
        _, info, _ = oracle.cg(A, M, b, rtol=RTOL, maxit=maxit)
    else:
        _, info, _ = oracle.gmres(A, M, b, restart=30, rtol=RTOL, maxit=maxit, flexible=w["solver"] == "fgmres")
    return time.perf_counter() - t0, info["iters"], o["clock"][0]


def oracle_run(w, A_host, xt, maxit, net_file=NET_PATH, net_slab=None):
    """Setup and one solve: (solve seconds, setup seconds, iterations, seconds
    of the solve spent in the network, network volume factor)."""
    o = oracle_setup(w, A_host, xt, net_file, net_slab)
    t, it, tnet = oracle_solve(o, w, maxit)
    return t, o["setup"], it, tnet, o["vol"]


def load_net_host(path):
    """Parameters and output scale from a checkpoint file (header, then FP32 arrays)."""
    import struct
    with open(path, "rb") as f:
        raw = f.read()
    magic, version, nparams, out_scale, step = struct.unpack("<IiqfI", raw[:24])
    flat = np.frombuffer(raw[24:24 + 4 * nparams], dtype=np.float32)
    from paper_1701_05913_gb300 import net_unflatten
    return net_unflatten(flat), float(out_scale)


# z-planes the numpy network covers in a timing sample of the learned
# stage (its time is then scaled by nz / planes): the CPU baseline of the
# bench line, and each step of the reference arm
NET_SLAB = {"bsr_learned": 16}
NET_SLAB_REF = {"bsr_learned": 8}
# iteration counts of the GPU solves, taken by the reference arm, which
# does not run the GPU (a full oracle solve of these systems takes minutes
# to hours on one core)
GPU_ITERS = {"learned": 26, "bsr": 30, "bsr_learned": 32}
# iterations an oracle sample runs on systems too large for a full solve
SAMPLE_ITERS = {"learned": 1, "bsr": 6, "bsr_learned": 1}


def _sample_words(w, o, slab):
    if w["precond"] != "cpr_learned":
        return ""
    nx, ny, nz = w["grid"]
    what = " with the numpy network (bf16-rounded) as the pressure stage"
    if slab is not None and o["vol"] != 1.0:
        what += (", the network run on a %dx%dx%d slab of the grid and its time scaled by %g (it is fully "
                 "convolutional: cost proportional to voxels)" % (nx, ny, nz / o["vol"], o["vol"]))
    return what


def oracle_baseline(w, A_host, xt, gpu_iters, slab_table=NET_SLAB, o=None):
    """The oracle's solve time (setup excluded, as in the GPU arm's steps) on
    one host core: a full solve where that takes seconds, else a bounded
    sample of iterations scaled to the iteration count."""
    n = A_host["n"] if "n" in A_host else 3 * A_host["nb"]
    slab = slab_table.get(w["kind"])
    if o is None:
        o = oracle_setup(w, A_host, xt, net_slab=slab)
    if w["kind"] == "csr" and n <= 1_100_000:
        t, it, _ = oracle_solve(o, w, 10000)
        return {"value": t, "unit": "s", "cores": 1, "kind": "oracle",
                "sample": "one full solve of the same system on one host core (%d iterations; setup %.3f s, not "
                          "included)" % (it, o["setup"])}
    t, it, tnet = oracle_solve(o, w, SAMPLE_ITERS.get(w["kind"], 30))
    per_it = ((t - tnet) + tnet * o["vol"]) / max(it, 1)
    return {"value": per_it * gpu_iters, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": "%d iteration(s) of the same solve%s on one host core (%.2f s per iteration), scaled to %s "
                      "iterations (setup %.2f s, not included)" % (it, _sample_words(w, o, slab), per_it, gpu_iters,
                                                                  o["setup"])}


# z-planes of the sub-grid a reference-arm step samples on the largest
# systems: one iteration there, its time scaled by the volume (every part
# of an iteration costs in proportion to the unknowns), so that the arm's
# steps stay within minutes
REF_SLAB_Z = {"bsr_learned": 16}


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    grid0 = w["grid"]
    zs = REF_SLAB_Z.get(w["kind"])
    vscale = 1.0
    if zs is not None and zs < w["grid"][2]:
        vscale = w["grid"][2] / zs
        w = dict(w, grid=(w["grid"][0], w["grid"][1], zs))
    g, A_host, xt = host_problem(w, w.get("seeds", [SEED])[0])
    o = oracle_setup(w, A_host, xt, net_slab=None if zs is not None else NET_SLAB_REF.get(w["kind"]))
    per = []
    if w["kind"] == "csr":
        full_t, full_it, _ = oracle_solve(o, w, 10000)
        for s in range(max(args.warmup - 1, 0) + args.steps):
            t, done, _ = oracle_solve(o, w, 30)
            if s >= args.warmup - 1:
                per.append(t / done * full_it)
        sample = ("one full solve (%d iterations, %.2f s) then, per step, 30 iterations of the same solve "
                  "scaled to %d iterations (setup %.2f s, once, not included)" % (full_it, full_t, full_it,
                                                                                  o["setup"]))
    else:
        cb = None
        for s in range(args.warmup + args.steps):
            cb = oracle_baseline(w, A_host, xt, GPU_ITERS[w["kind"]], NET_SLAB_REF, o=o)
            if s >= args.warmup:
                per.append(cb["value"] * vscale)
        sample = cb["sample"] + " (iteration count of the GPU arm's solve assumed)"
        if vscale != 1.0:
            sample = ("on the %dx%dx%d sub-grid of the same generator, scaled by the volume %g: " %
                      (tuple(w["grid"]) + (vscale,))) + sample
    v = statistics.mean(per)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if w["prec"] == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(grid0), "solver": w["solver"],
                   "precond": w["precond"], "precision": w["prec"], "rtol": RTOL},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks of the default
    process group (a no-op without one); used for the slowest-rank timing."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
class Case:
    """One resident problem: matrix, right-hand side, preconditioner(s)."""

    def __init__(self, rs, ctx, w, seed, net=None):
        g, A_host, xt = host_problem(w, seed)
        self.g, self.A_host = g, A_host
        self.xt = xt
        if w["kind"] in ("bsr", "bsr_learned"):
            self.A = rs.Mat.bsr(ctx, A_host)
        else:
            self.A = rs.Mat.csr(ctx, A_host)
        n = self.A.n
        self.b = rs.Vec.zeros(ctx, n)
        self.A.spmv(rs.Vec(ctx, xt), self.b)
        self.x = rs.Vec.zeros(ctx, n)
        ctx.sync()
        t0 = time.perf_counter()
        kw = dict(form=w["form"]) if "form" in w else {}
        if w["precond"] == "cpr_learned":
            kw.update(net=net, log_perm=A_host["logk"], grid=w["grid"])
        if "ras" in w:
            kw.update(ras_kwargs(w))
        if "amg" in w:
            kw.update(amg=w["amg"], **({"pstage": w["pstage"]} if "pstage" in w else {}))
        self.M = rs.Precond(ctx, self.A, w["precond"], prec=w["prec"], **kw)
        ctx.sync()
        self.setup_s = time.perf_counter() - t0
        self.Mbase = None
        if w["kind"] == "learned":
            self.Mbase = rs.Precond(ctx, self.A, "ilu0", prec=w["prec"])
        elif w["kind"] == "bsr_learned":
            self.Mbase = rs.Precond(ctx, self.A, "cpr", prec=w["prec"])
        ctx.sync()


def solve_fn(rs, w):
    if w["solver"] == "bicgstab":
        return lambda c, M: rs.solve_bicgstab(c.A, M, c.b, c.x, rtol=RTOL)
    if w["solver"] == "cg":
        return lambda c, M: rs.solve_cg(c.A, M, c.b, c.x, rtol=RTOL)
    if w["solver"] == "fgmres":
        return lambda c, M: rs.solve_fgmres(c.A, M, c.b, c.x, restart=30, rtol=RTOL)
    if w["solver"] == "lgmres":
        return lambda c, M: rs.solve_lgmres(c.A, M, c.b, c.x, restart=30, aug_k=w["aug_k"], rtol=RTOL)
    return lambda c, M: rs.solve_gmres(c.A, M, c.b, c.x, restart=30, rtol=RTOL)


def run_gpu(args, w, rank, world, local):
    import torch

    import paper_1701_05913_gb300 as rs

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ctx = rs.Context(local)
    stream = torch.cuda.current_stream()
    net = rs.Net(ctx, path=NET_PATH) if w["precond"] == "cpr_learned" else None
    seeds = w.get("seeds", [SEED])
    cases = [Case(rs, ctx, w, s, net) for s in seeds]
    solve = solve_fn(rs, w)
    base_solve = (lambda c, M: rs.solve_gmres(c.A, M, c.b, c.x, restart=30, rtol=RTOL)) if w["kind"] == "learned" \
        else solve

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for s in range(args.warmup):
        c = cases[s % len(cases)]
        c.x.t.zero_()
        solve(c, c.M)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fn_pick, profile):
        evs, infos = [], []
        for s in range(args.steps):
            c = cases[s % len(cases)]
            c.x.t.zero_()
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(fn_pick(c))
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs], infos

    # the headline: K steps with the library's profiler off (its per-kernel
    # events would add time and keep the AMG V-cycles out of CUDA graphs),
    # clocks sampled meanwhile
    clocks = ClockSampler(local)
    clocks.start()
    n_launch0 = ctx.launches()
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms, infos = timed(lambda c: solve(c, c.M), False)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    launches = ctx.launches() - n_launch0
    clk = clocks.stop()
    ms = sum(step_ms) / len(step_ms)
    # then the same K steps with the profiler on, for the per-kernel classes
    # behind the roofline object
    ctx.prof_enable(True)
    ctx.prof_read(reset=True)
    step_ms2, _ = timed(lambda c: solve(c, c.M), True)
    prof = ctx.prof_read(reset=True)
    ctx.prof_enable(False)
    ms_prof = sum(step_ms2) / len(step_ms2)
    base = None
    if cases[0].Mbase is not None:
        bms, binfos = timed(lambda c: base_solve(c, c.Mbase), False)
        base = {"value": sum(bms) / len(bms) / 1e3, "unit": "s",
                "method": "GMRES(30)+ILU(0)" if w["kind"] == "learned" else "FGMRES(30)+CPR with ILU(0) pressure stage",
                "iters": statistics.median(i["iters"] for i in binfos),
                "true_rel_res": max(i["true_rel_res"] for i in binfos)}

    # end to end through the C ABI: b from pinned host memory, x back to pinned host memory
    L = rs.lib()
    e2e = []
    hbs = [torch.from_numpy(c.b.numpy()).pin_memory() for c in cases]
    hx = torch.empty(cases[0].A.n, dtype=torch.float64).pin_memory()
    for s in range(args.steps):
        c = cases[s % len(cases)]
        c.x.t.zero_()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.rs_vec_set(c.b.h, rs._vp(hbs[s % len(cases)].data_ptr()), rs.MEM_HOST)
        solve(c, c.M)
        L.rs_vec_get(c.x.h, rs._vp(hx.data_ptr()), rs.MEM_HOST)
        e2e.append(time.perf_counter() - t1)
    # the same statistic as the device-timed value (the mean of the K steps)
    e2e_s = statistics.mean(e2e)

    if world > 1:
        ms, ms_prof, e2e_s, wall = max_over_ranks([ms, ms_prof, e2e_s, wall], device="cuda")

    # roofline of the dominant kernel class, from the live profile
    hbm, bf16, peak_src = measured_peaks()
    model, nunk = kernel_model(w, cases[0].A_host, cases[0].M.ras_info() if "ras" in w else None)
    iters = [i["iters"] for i in infos]
    cb = cgs_bytes(nunk, iters)
    kern_ms = {k: v[0] for k, v in prof.items() if v[1] > 0}
    kern_n = {k: v[1] for k, v in prof.items() if v[1] > 0}
    total_prof = sum(kern_ms.values())
    amg_vc = amg_vcycle_model(w, cases[0].M.amg_sizes()) if "amg" in w else None
    done = executed_launches(w, infos, amg_vc, model["spmv"])
    work = {k: model[k] * done[k] for k in model if k in kern_n and done.get(k)}
    if amg_vc and "spmv" in work:
        work["spmv"] = done["_spmv_bytes"]
    work.update({k: cb[k] for k in cb if k in kern_n})
    rate = {k: work[k] / (kern_ms[k] * 1e-3) / 1e9 for k in work}
    cf = cgs_fmas(nunk, iters)
    fma_rate = {k: cf[k] / (kern_ms[k] * 1e-3) for k in cf if k in kern_n}
    net_fl = None
    if "net" in kern_n and net is not None:
        net_fl = net_flops(w["grid"]) * done["net"] / (kern_ms["net"] * 1e-3) / 1e12
    dom = max(kern_ms, key=kern_ms.get)
    if dom in fma_rate:
        roofline = {"kernel": dom, "bound": "fp64", "achieved": round(fma_rate[dom] / 1e9, 2),
                    "peak": FP64_FMA_PEAK / 1e9, "unit": "G FMA/s", "frac": round(fma_rate[dom] / FP64_FMA_PEAK, 4),
                    "traffic": ncu_traffic(dom, args.workload), "peak_source": "nominal FP64 rate"}
    elif dom == "net":
        roofline = {"kernel": "net (all U-Net kernels of one pressure-stage apply)", "bound": "tensor",
                    "achieved": round(net_fl, 2), "peak": bf16, "unit": "TFLOP/s", "frac": round(net_fl / bf16, 4),
                    "traffic": ncu_traffic("net", args.workload), "peak_source": peak_src,
                    "alg_flops_per_launch": net_flops(w["grid"])}
    else:
        roofline = {"kernel": dom, "bound": "hbm", "achieved": round(rate.get(dom, 0.0), 2), "peak": hbm,
                    "unit": "GB/s", "frac": round(rate.get(dom, 0.0) / hbm, 4),
                    "traffic": ncu_traffic(dom, args.workload), "peak_source": peak_src,
                    "alg_bytes_per_launch": int(work.get(dom, 0) / max(done.get(dom, kern_n[dom]), 1)),
                    "avg_launch_us": round(kern_ms[dom] / max(done.get(dom, kern_n[dom]), 1) * 1e3, 2),
                    "launches_with_work": done.get(dom, kern_n[dom]), "launches_total": kern_n[dom]}
    roofline["share_of_kernel_time"] = round(kern_ms[dom] / total_prof, 3)
    if dom in ("l_sweep", "u_sweep", "bl_sweep", "bu_sweep") and \
            dom.startswith("b") == (w["kind"] in ("bsr", "bsr_learned")):
        # the sweeps are bound by their dependency chain, not by bytes: its
        # length (wavefront cells nx + ny + nz - 2, or segment levels) and
        # the time per step of it
        lv = cases[0].M.sweep_levels()[0 if dom in ("l_sweep", "bl_sweep") else 1]
        kind = cases[0].M.sweep_kind()[0]
        roofline["critical_path"] = {"kind": "wavefront cells" if kind == "wavefront" else "segment levels",
                                     "length": lv, "us_per_step": round(roofline["avg_launch_us"] / lv, 4)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        c0 = cases[0]
        cpu = oracle_baseline(w, c0.A_host, c0.xt, statistics.median(iters))

    if rank == 0:
        ilu_k = [k for k in ("l_sweep", "u_sweep", "bl_sweep", "bu_sweep") if k in work]
        line = {
            "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if w["prec"] == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "grid": list(w["grid"]), "unknowns": cases[0].A.n,
                       "nnz": int(cases[0].A.nnz), "block_size": cases[0].A.bs,
                       "solver": w["solver"] + ("(30,%d)" % w["aug_k"] if "aug_k" in w else "(30)")
                       if "gmres" in w["solver"] else w["solver"],
                       "precond": w["precond"] + ("-" + w["form"] if "form" in w else "")
                       + ("+amg" if w.get("pstage") == "amg" else "")
                       + ("+ras" if "ras" in w and w["precond"] != "ras" else ""),
                       "precision": w["prec"], "rtol": RTOL, "seeds": [seeds[0], seeds[-1]],
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": "replicas" if world > 1 else "1 gpu",
                       **({"ras": dict(w["ras"], stacked_rows=cases[0].M.ras_info()[0])} if "ras" in w else {})},
            "iters": statistics.median(iters),
            "true_rel_res": max(i["true_rel_res"] for i in infos),
            "setup_s": statistics.median(c.setup_s for c in cases),
            "ms_per_step_with_profiler": ms_prof,
            "wall_s": wall,
            "baseline_method": base,
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * cases[0].A.n,
                    "d2h_bytes_per_step": 8 * cases[0].A.n},
            "gpu_launches": launches,
            "roofline": roofline,
            "kernels": {k: {"ms_per_step": round(kern_ms[k] / args.steps, 4),
                            "launches_per_step": kern_n[k] / args.steps,
                            **({"launches_with_work_per_step": done[k] / args.steps} if k in done else {}),
                            "share": round(kern_ms[k] / total_prof, 4),
                            **({"GBs": round(rate[k], 1)} if k in rate else {}),
                            **({"GFMAs": round(fma_rate[k] / 1e9, 1),
                                "fp64_frac": round(fma_rate[k] / FP64_FMA_PEAK, 3)} if k in fma_rate else {}),
                            **({"TFLOPs": round(net_fl, 2)} if k == "net" and net_fl else {})} for k in kern_ms},
            "spmv_GBs": round(rate.get("spmv", 0.0), 1),
            "ilu_apply_GBs": round(sum(work[k] for k in ilu_k) / (sum(kern_ms[k] for k in ilu_k) * 1e-3) / 1e9, 1)
            if ilu_k else None,
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
    if args.grid:
        w = dict(w, grid=tuple(int(v) for v in args.grid.split(",")))
        if len(w["grid"]) != 3 or min(w["grid"]) < 1:
            raise SystemExit("--grid wants NX,NY,NZ")
        args.workload = "%s@%dx%dx%d" % ((args.workload,) + w["grid"])
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    run_gpu(args, w, rank, world, local)


if __name__ == "__main__":
    main()
