"""Benchmark: time to a 1e-10 relative residual (hence backward error <= 1e-10)
of mixed-precision GADI (FP64 outer, FP32 inner) against plain FP64 GADI on
the same GPU, on 2D convection-diffusion -Lap u + beta.grad u, 5-point
centred differences on a 2048 x 2048 interior grid (n = 4,194,304), beta drawn
from U[1,100]^2 by seed, b = A x_true with x_true ~ U[0,1).

One step = one complete mixed-precision solve from x_0 = 0 to the tolerance
(every step of Algorithm 1: residual, H-solve, S-solve, update, stopping
test), inputs resident in HBM, timed with CUDA events on the solve's stream.
The L2 cache is flushed (a 256 MB buffer is written) before each step.
Printed as one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (a bounded sample, see `cpu_baseline`).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "conv-diff-2d 2048x2048 (n=4194304), beta~U[1,100]^2 seed 2, HSS, tol 1e-10"
# GADI parameters shared by the mixed and the plain FP64 runs
ALPHA_FACTOR = 8.0     # alpha = ALPHA_FACTOR * alpha* (closed-form HSS value)
OMEGA = 0.0
TOL = 1e-10
MAXIT = 20000
TOL_INNER = 1e-3       # default inner tolerance (other configurations)
# 2048^2 inner tolerances, shared by the mixed and the FP64 runs: 1e-2 on the
# H-solve was faster for FP32 but let plain FP64 GADI stagnate, so both use 1e-3
TOL_H, TOL_S = 1e-3, 1e-3
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "kernel_traffic.json")
KERNEL_SOURCES = ["gadi_kernel.cuh", "gadi_solver.cuh", "gadi_common.cuh", "gadi_params.h",
                  "gadi_inst_2d5.cu", "gadi_inst_2d5r.cu", "gadi_inst_2d5t.cu"]


# stats["h_resident"]: the form the CG on H took
H_SOLVE = {0: "streaming", 1: "p in shared memory", 2: "p in shared memory, z and r in tensor memory"}


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2512_21164_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record() -> dict:
    try:
        with open(TRAFFIC_RECORD) as f:
            return json.load(f)
    except Exception:
        return {}


def measured_traffic(alg_bytes: float):
    """DRAM bytes of one launch from the committed ncu record (DRAM bytes per
    algorithmic byte of a capped solve of the same kernel, scaled to this
    launch), or None if the kernel sources changed since the capture."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
        if rec.get("kernel_source_hash") != kernel_source_hash():
            return None
        return rec["dram_bytes_per_algorithmic_byte"] * alg_bytes
    except Exception:
        return None
HBM_FALLBACK = 6800.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.p = None
        self.out = ""

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        # wait (3 s at most) for the first sample, taken before the timed
        # region: nvidia-smi's start-up can hold up the CUDA calls that
        # launch a step, which the step's events would then count
        if self.p is not None:
            import select
            if select.select([self.p.stdout], [], [], 3.0)[0]:
                self.p.stdout.readline()
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(n: int, stats: dict, s_bytes: int, d_bytes: int = 8) -> float:
    """Bytes the method must move for one solve (per point: outer residual +
    update 3d+2s, each CG iteration on H 8s, each CGNR iteration on S 8s, the
    CGNR set-up S^T g 2s)."""
    k = stats["outer_its"]
    per_pt = (k + 1) * (3 * d_bytes + 2 * s_bytes) + 8 * s_bytes * (stats["inner_its_h"] + stats["inner_its_s"]) \
        + 2 * s_bytes * k
    return float(n) * per_pt


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import alpha_star, config2

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    B.build()
    p, xt = config2(args.grid)
    alpha = ALPHA_FACTOR * alpha_star(p)
    n = p.nvec
    H = G.Gadi.from_problem(p)
    stream = torch.cuda.current_stream()
    xtd = torch.from_numpy(xt).cuda()
    b = torch.zeros_like(xtd)
    H.apply(G.OP_A, xtd, b)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    kw = dict(tol_h=TOL_H, tol_s=TOL_S)

    def one(prec):
        x.zero_()
        flush.zero_()
        st, s = H.solve(b, x, alpha, OMEGA, prec, TOL, args.maxit, **kw)
        return st, s

    for _ in range(args.warmup):
        one(G.FP32)
    # timed region: K mixed-precision solves
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_s, per = [], []
    with Clocks(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.time()
        for _ in range(args.steps):
            flush.zero_()
            x.zero_()
            ev0.record(stream)
            st, s = H.solve(b, x, alpha, OMEGA, G.FP32, TOL, args.maxit, **kw)
            ev1.record(stream)
            torch.cuda.synchronize()
            per.append(ev0.elapsed_time(ev1) / 1e3)
            kern_s.append(s["seconds"])
        torch.cuda.synchronize()
        t_wall = time.time() - t_wall
    if world > 1:
        t = torch.tensor([max(per)], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    mixed_stats, mixed_status = s, st
    # check the answer: FP64 residual through the library's own operator
    r = torch.zeros_like(b)
    H.apply(G.OP_A, x, r)
    relres = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
    anorm = H.norm2(50)
    be = float(torch.linalg.norm(b - r) / (anorm * torch.linalg.norm(x) + torch.linalg.norm(b)))
    fe = float(torch.linalg.norm(x - xtd) / torch.linalg.norm(xtd))

    # plain FP64 GADI on the same GPU, same alpha/omega/tolerances
    fp64 = None
    if not args.skip_fp64:
        one(G.FP64)  # warm-up
        f_times = []
        for _ in range(args.fp64_steps):
            flush.zero_()
            x.zero_()
            ev0.record(stream)
            st64, s64 = H.solve(b, x, alpha, OMEGA, G.FP64, TOL, args.maxit, **kw)
            ev1.record(stream)
            torch.cuda.synchronize()
            f_times.append(ev0.elapsed_time(ev1) / 1e3)
        H.apply(G.OP_A, x, r)
        fp64 = {"seconds": statistics.median(f_times), "step_s": f_times, "status": G.status_str(st64),
                "outer_its": s64["outer_its"], "inner_its_h": s64["inner_its_h"],
                "inner_its_s": s64["inner_its_s"],
                "relres": float(torch.linalg.norm(b - r) / torch.linalg.norm(b)),
                "kernel_GBps": algorithmic_bytes(n, s64, 8) / s64["seconds"] / 1e9}

    # what binds the mixed kernel: its grid-wide sums (two per CG or CGNR
    # iteration, one per CGNR set-up and per z/y hand-over) and the FP64
    # residual step, each measured on its own
    t_sum = G.probe_sync(0, 20000) * 1e-6
    y0 = torch.zeros(n, dtype=torch.float32, device="cuda")
    xo = torch.empty_like(b)
    rs = torch.empty(n, dtype=torch.float32, device="cuda")
    for _ in range(3):
        H.step_residual(G.FP32, b, x, y0, xo, None, rs)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(20):
        H.step_residual(G.FP32, b, x, y0, xo, None, rs)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_res = ev0.elapsed_time(ev1) / 1e3 / 20
    fp64_gops, fp64_per_clk = G.probe_fp64()

    # end-to-end through the C ABI with host (pinned) buffers
    bh = b.cpu().pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e = []
    for i in range(max(1, min(args.steps, 2))):
        flush.zero_()
        xh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H.solve(bh.numpy(), xh.numpy(), alpha, OMEGA, G.FP32, TOL, args.maxit, **kw)
        e2e.append(time.perf_counter() - t0)

    hbm, src = _peaks()
    value = statistics.mean(per)
    ab = algorithmic_bytes(n, mixed_stats, 4)
    kmean = statistics.mean(kern_s)
    achieved = ab / kmean / 1e9
    k_out = mixed_stats["outer_its"]
    n_sums = 2 * (mixed_stats["inner_its_h"] + mixed_stats["inner_its_s"]) + 3 * k_out
    floor_s = n_sums * t_sum + (k_out + 1) * t_res
    traffic = measured_traffic(ab)
    rec = traffic_record()
    latency = {
        "grid_sum_us": t_sum * 1e6, "grid_sums": n_sums, "residual_step_ms": t_res * 1e3,
        "floor_s": floor_s, "kernel_s": kmean, "kernel_over_floor": kmean / floor_s,
        "note": "floor = grid sums x measured time of one (gadi_probe_sync, 152 blocks) + outer iterations x "
                "measured FP64 residual step (gadi_step_residual launched alone, launch included); the rest of "
                "the kernel time is the inner sweeps over vectors held in shared memory, tensor memory and L2"}
    if fp64 is not None:
        # GADI-FP64: FP64 pipe operations (an FMA counts one) the method's
        # definition needs per grid point: residual 8 (x + y, A x in 5,
        # b - A x, r.r), CG iteration 10 (p update, H p in 5, p.Hp, z, r,
        # r.r), CGNR iteration 15 (p, S p in 5, u.u, S^T u in 5, y, t, t.t),
        # CGNR set-up 7 (g, S^T g in 5, t.t)
        ops = n * (8 * (fp64["outer_its"] + 1) + 10 * fp64["inner_its_h"] + 15 * fp64["inner_its_s"]
                   + 7 * fp64["outer_its"])
        fp64["fp64_pipe"] = {"ops": ops, "achieved_gops": ops / fp64["seconds"] / 1e9,
                             "peak_gops": fp64_gops, "frac": ops / fp64["seconds"] / 1e9 / fp64_gops,
                             "peak_fma_per_sm_clk": fp64_per_clk,
                             "peak_source": "measured (gadi_probe_fp64: 8 independent FMA chains per thread)"}
    out = {
        "metric": "time to 1e-10 rel. backward error: mixed vs FP64 GADI, 1 GB300; HBM %peak",
        "value": value, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 outer / f32 inner", "data": "synthetic",
        "config": {"workload": WORKLOAD, "alpha": alpha, "alpha_over_alpha_star": ALPHA_FACTOR,
                   "omega": OMEGA, "tol_h": TOL_H, "tol_s": TOL_S, "u_s": "fp32", "u": "fp64",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "flushed (256 MB write) before each step"},
        "status": G.status_str(mixed_status), "outer_its": mixed_stats["outer_its"],
        "inner_its_h": mixed_stats["inner_its_h"], "inner_its_s": mixed_stats["inner_its_s"],
        "relres": relres, "backward_error": be, "forward_error": fe,
        "fp64_plain": fp64,
        "speedup_vs_fp64": (fp64["seconds"] / value) if fp64 else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": src,
                     "dram_gbs": traffic / kmean / 1e9 if traffic else None,
                     "l2_throughput_pct": rec.get("l2_throughput_pct") if traffic else None,
                     "latency": latency,
                     "kernel": "gadi_stencil_kernel<2D5,FP32> (persistent, one launch per solve; H-solve: "
                               + H_SOLVE[mixed_stats["h_resident"]] + "; S-solve: "
                               + ("p in shared memory, t and y in tensor memory" if mixed_stats.get("s_resident")
                                  else "streaming") + ")",
                     "algorithmic_bytes": ab},
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": 2 * 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
        "wall_s": t_wall,
        "step_s": per,
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_profile_case(args):
    """A small, bounded launch for ncu: one solve of the benchmark workload
    (or, with --workload c3, of the 3D workload at --grid3) capped at --maxit
    outer iterations (the first kernel launch is the FP64 operator
    application that forms b; the solve is the second)."""
    import torch

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import alpha_star, config2
    B.build()
    prec = {"fp64": G.FP64, "fp32": G.FP32, "bf16": G.BF16}[args.profile_case]
    omega = OMEGA
    if args.workload == "c3":
        from workloads import config3
        p, xt = config3(args.grid3)
        omega = OMEGA if args.omega is None else args.omega
    elif args.workload == "c4":
        from workloads import config4
        p, xt = config4(args.grid4)
        omega = 1.0
    else:
        p, xt = config2(args.grid)
    Hs = G.Gadi.from_problem(p)
    xtd = torch.from_numpy(xt).cuda()
    b = torch.zeros_like(xtd)
    Hs.apply(G.OP_A, xtd, b)
    x = torch.zeros_like(b)
    if args.workload == "csr2d":
        # the same matrix assembled as CSR (the solve is then the third launch)
        from workloads import K_CSR, Problem
        rp, cl, vl = G.stencil_csr(p)
        H = G.Gadi.from_problem(Problem(K_CSR, p.npoints, rowptr=rp, col=cl, val=vl))
    else:
        H = Hs
    af = {"c3": args.alpha_factor, "c4": 1.0}.get(args.workload, ALPHA_FACTOR)
    tin = 1e-2 if prec == G.BF16 else TOL_H
    st, s = H.solve(b, x, af * alpha_star(p), omega, prec, TOL, args.maxit, tol_h=tin, tol_s=tin)
    print(json.dumps({"profile_case": args.profile_case, "status": G.status_str(st), **s}))


def record_traffic(rep: str, case_log: str):
    """Write the traffic record from an ncu report of the --profile-case solve
    launch (dram__bytes_read.sum + dram__bytes_write.sum, read with `ncu -i`,
    no GPU needed) and that run's JSON line (its iteration counts give the
    launch's algorithmic bytes)."""
    import csv
    import subprocess
    with open(case_log) as f:
        stats = [json.loads(l) for l in f if l.startswith("{")][-1]
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    head, units, vals = rows[0], rows[1], rows[-1]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    got = {}
    for k, u, v in zip(head, units, vals):
        if k in ("dram__bytes_read.sum", "dram__bytes_write.sum", "Kernel Name", "gpu__time_duration.sum",
                 "lts__throughput.avg.pct_of_peak_sustained_elapsed",
                 "gpu__compute_memory_throughput.avg.pct_of_peak_sustained_elapsed"):
            got[k] = (v, u)
    dram = sum(float(got[k][0].replace(",", "")) * scale[got[k][1]]
               for k in ("dram__bytes_read.sum", "dram__bytes_write.sum"))
    from workloads import config2
    p, _ = config2()
    sb = {"fp64": 8, "fp32": 4, "bf16": 2}[stats["profile_case"]]
    alg = algorithmic_bytes(p.npoints, stats, sb)
    rec = {"kernel": got["Kernel Name"][0], "case": f"--profile-case {stats['profile_case']}",
           "outer_its": stats["outer_its"], "inner_its_h": stats["inner_its_h"],
           "inner_its_s": stats["inner_its_s"], "dram_bytes": dram, "algorithmic_bytes": alg,
           "dram_bytes_per_algorithmic_byte": dram / alg, "kernel_source_hash": kernel_source_hash(),
           "l2_throughput_pct": float(got["lts__throughput.avg.pct_of_peak_sustained_elapsed"][0].replace(",", ""))
           if "lts__throughput.avg.pct_of_peak_sustained_elapsed" in got else None,
           "source": f"ncu -i {os.path.basename(rep)} (dram__bytes_read.sum + dram__bytes_write.sum)"}
    with open(TRAFFIC_RECORD, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


# Other configurations: the same measurement, one JSON line per precision.
# Not the default headline line (that is the 2048^2 default above).
WORKLOADS = {
    # name: (builder, precisions, alpha factor, omega, maxit, inner tol per precision)
    "c1": ("conv-diff-2d 64x64, beta=(10,10), alpha=0.5, omega=1, maxit 500, plain FP64", ["fp64"]),
    "c3": ("conv-diff-3d 512^3 (n=134217728), beta=(1,1,1)U[1,50] seed 3", ["bf16", "fp32", "fp64"]),
    "c2s": (WORKLOAD + ", alpha = alpha*, omega = 1 (the untuned closed-form choice)", ["fp32", "fp64"]),
    "c4": ("complex reaction-diffusion 4096^2 (n=16777216 complex), kappa~U[0,10], sigma~U[1,100] seed 4",
           ["bf16", "fp32", "fp64"]),
}


# The paper's own A100 runtimes (seconds; FP64, FP32, BF16 inner precision)
# for its problem instances, as printed in its Tables 2 (2D CDR, tolerance
# 1e-10) and 3 (3D CD, tolerance 1e-6): context for the same instances here,
# not a like-for-like target (another GPU, and alpha from the paper's GPR).
PAPER_TABLE2 = {960: (4.9, 5.1, 3.6), 2560: (44.3, 31.5, 19.9), 4096: (121.0, 84.0, 58.6),
                8192: (768.1, 444.6, 307.2), 10000: (1373.0, 779.2, 529.5)}
PAPER_TABLE3 = {180: (3.9, 2.4, 2.8), 256: (12.2, 7.3, 8.9), 320: (25.7, 15.3, 18.4), 360: (40.2, 23.9, 26.4),
                400: (62.7, 36.9, 50.3), 450: (101.1, 60.6, 137.3), 512: (None, None, 390.7)}
# Table 4 (complex reaction-diffusion, tolerance 1e-6)
PAPER_TABLE4 = {1024: (6.2, 4.0, 2.4), 2048: (21.8, 13.1, 8.1), 4096: (79.6, 46.5, 27.7),
                5120: (121.7, 72.4, 40.2), 8192: (309.0, 180.2, 98.7)}


def run_paper(args):
    """The paper's own instances (Sec. 5.2 2D CDR at tolerance 1e-10, Sec. 5.3
    3D CD and Sec. 5.4 complex RD at 1e-6; b from x = ones), at its grid sizes, every inner precision,
    alpha = f alpha* and omega for each pair in --alpha-factors (the paper
    picks alpha by GPR; the fastest pair is reported).  One JSON line per
    (grid, precision) with the paper's A100 time beside ours."""
    import torch

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import alpha_star, paper_cd_3d, paper_cdr_2d, paper_complex_rd
    B.build()
    w = args.workload
    grids = [int(v) for v in args.grids.split(",")] if args.grids else \
        {"paper2d": [960, 2560, 4096], "paper3d": [180, 256, 320], "paperc": [1024, 2048, 4096]}[w]
    spec = args.alpha_factors or {"paper2d": "4:0,8:0,16:0", "paper3d": "0.05:1,0.1:1,0.3:1",
                                  "paperc": "64:1,256:1,1024:1"}[w]
    gpr = spec.startswith("gpr")
    if gpr:
        # Sec. 4.2: alpha predicted by a GPR trained on small instances of the
        # family (sizes below), omega as given after the colon (default 0)
        omega_g = float(spec.split(":")[1]) if ":" in spec else 0.0
        train_sizes = {"paper2d": [64, 96, 128, 192], "paper3d": [24, 32, 48, 64],
                       "paperc": [64, 96, 128, 192]}[w]
        from paper_2512_21164_gb300 import alpha_gpr
        models = {}
        factors = []
    else:
        factors = [(float(v.split(":")[0]), float(v.split(":")[1]) if ":" in v else 0.0) for v in spec.split(",")]
    tol = 1e-10 if w == "paper2d" else 1e-6
    table = {"paper2d": PAPER_TABLE2, "paper3d": PAPER_TABLE3, "paperc": PAPER_TABLE4}[w]
    section = {"paper2d": "2D CDR (Sec. 5.2)", "paper3d": "3D CD (Sec. 5.3)", "paperc": "complex RD (Sec. 5.4)"}[w]
    for n in grids:
        p, xt = {"paper2d": paper_cdr_2d, "paper3d": paper_cd_3d, "paperc": paper_complex_rd}[w](n)
        H = G.Gadi.from_problem(p)
        xtd = torch.from_numpy(xt).cuda()
        b = torch.zeros_like(xtd)
        H.apply(G.OP_A, xtd, b)
        x = torch.zeros_like(b)
        a0 = alpha_star(p)
        for j, pn in enumerate(["fp64", "fp32", "bf16"]):
            if pn not in args.precs.split(","):
                continue
            prec = {"fp64": G.FP64, "fp32": G.FP32, "bf16": G.BF16}[pn]
            tin = 1e-2 if pn == "bf16" else TOL_INNER
            runs = []
            gpr_note = None
            if gpr:
                if pn not in models:
                    fam = {"paper2d": paper_cdr_2d, "paper3d": paper_cd_3d, "paperc": paper_complex_rd}[w]
                    models[pn] = alpha_gpr.train(fam, train_sizes, prec, omega_g, tol, alpha_star)
                fl, fs = models[pn].predict_log2_factor(n)
                factors = [(2.0 ** fl, omega_g)]
                gpr_note = {"log2_factor": fl, "std": fs, "train_sizes": train_sizes,
                            "train_best_log2": [float(v) for v in models[pn].gp.predict(models[pn].gp.x)[0]]}
            for f, om in factors:
                x.zero_()
                H.solve(b, x, f * a0, om, prec, tol, 3, tol_h=tin, tol_s=tin)  # warm-up
                x.zero_()
                st, s = H.solve(b, x, f * a0, om, prec, tol, args.maxit, tol_h=tin, tol_s=tin,
                                alpha_restarts=4)
                fe = float(torch.linalg.norm(x - xtd) / torch.linalg.norm(xtd))
                runs.append((st != G.OK, s["seconds"], (f, om), st, s, fe))
            runs.sort(key=lambda r: (r[0], r[1]))
            _, sec, (f, om), st, s, fe = runs[0]
            print(json.dumps({
                "metric": f"time to {tol:g} relative residual, the paper's {section} instance",
                "workload": args.workload, "grid": n, "n": p.nvec, "u_s": pn, "value": sec, "unit": "s",
                "status": G.status_str(st), "alpha_over_alpha_star": f, "alpha": s["alpha"], "omega": om,
                "outer_its": s["outer_its"], "inner_its_h": s["inner_its_h"], "inner_its_s": s["inner_its_s"],
                "restarts": s["restarts"], "relres": s["relres"], "forward_error": fe,
                "sweep": [{"f": r[2][0], "omega": r[2][1], "s": r[1], "status": G.status_str(r[3]),
                           "outer": r[4]["outer_its"]} for r in runs], "gpr": gpr_note,
                "paper_a100_s": table.get(n, (None, None, None))[j]}), flush=True)
        H.close()


def run_c2_dd(args):
    """The headline workload (2048^2, FP32 inner, alpha = 8 alpha*, omega = 0,
    tolerance 1e-10) with the residual in double-FP64 (u_r ~ u^2) beside the
    default FP64 residual: time, iterations, relres and forward error."""
    import torch

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import alpha_star, config2
    B.build()
    p, xt = config2(args.grid)
    H = G.Gadi.from_problem(p)
    xtd = torch.from_numpy(xt).cuda()
    b = torch.zeros_like(xtd)
    H.apply(G.OP_A, xtd, b)
    x = torch.zeros_like(b)
    alpha = ALPHA_FACTOR * alpha_star(p)
    for ur, name in ((G.FP64, "fp64"), (G.FP64X2, "double-fp64")):
        x.zero_()
        H.solve(b, x, alpha, OMEGA, G.FP32, TOL, 3, tol_h=TOL_H, tol_s=TOL_S, u_r=ur)  # warm-up
        x.zero_()
        st, s = H.solve(b, x, alpha, OMEGA, G.FP32, TOL, args.maxit, tol_h=TOL_H, tol_s=TOL_S, u_r=ur)
        fe = float(torch.linalg.norm(x - xtd) / torch.linalg.norm(xtd))
        print(json.dumps({
            "metric": "time to 1e-10 relative residual with residual precision u_r", "workload": "c2dd",
            "config": {"workload": WORKLOAD, "alpha_over_alpha_star": ALPHA_FACTOR, "omega": OMEGA,
                       "u_s": "fp32", "u_r": name},
            "value": s["seconds"], "unit": "s", "status": G.status_str(st), "outer_its": s["outer_its"],
            "inner_its_h": s["inner_its_h"], "inner_its_s": s["inner_its_s"], "relres": s["relres"],
            "forward_error": fe, "ms_per_outer": 1e3 * s["seconds"] / max(1, s["outer_its"])}), flush=True)


def run_workload(args):
    """Time-to-tolerance of one configuration for each precision (one solve
    each after a capped warm-up), with the same roofline accounting as the
    headline line.  Solves that need more than --maxit outer iterations end
    with their status reported; --fp64-maxit caps the slow FP64 runs (the
    line then reports the per-outer-iteration time, not a time to tolerance)."""
    import torch

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import alpha_star, config1, config3, config4
    B.build()
    name = args.workload
    desc, precs = WORKLOADS[name]
    if name == "c1":
        p, xt, c = config1()
        alpha, omega, maxit = c["alpha"], c["omega"], c["maxit"]
    elif name == "c2s":
        from workloads import config2
        p, xt = config2(args.grid)
        alpha, omega, maxit = alpha_star(p), 1.0, args.maxit
    elif name == "c3":
        p, xt = config3(args.grid3)
        alpha, maxit = args.alpha_factor * alpha_star(p), args.maxit
        omega = OMEGA if args.omega is None else args.omega
    else:
        p, xt = config4(args.grid4)
        alpha, omega, maxit = alpha_star(p), 1.0, args.maxit
    H = G.Gadi.from_problem(p)
    xtd = torch.from_numpy(xt).cuda()
    b = torch.zeros_like(xtd)
    H.apply(G.OP_A, xtd, b)
    x = torch.zeros_like(b)
    r = torch.zeros_like(b)
    hbm, src = _peaks()
    dbytes = 16 if p.kind == 2 else 8
    for pn in [q for q in precs if q in args.precs.split(",")]:
        prec = {"fp64": G.FP64, "fp32": G.FP32, "bf16": G.BF16}[pn]
        sbytes = {"fp64": 8, "fp32": 4, "bf16": 2}[pn] * (2 if p.kind == 2 else 1)
        tin = 1e-2 if pn == "bf16" else TOL_INNER
        mit = min(maxit, args.fp64_maxit) if pn == "fp64" and name != "c1" else maxit
        a_run = alpha
        if args.alpha_select and name != "c1":
            # Sec. 4.3: the smallest alpha * 2^k with kappa(H) kappa(S) u_s < tau
            a_run = G.select_alpha(p, alpha, prec, args.tau)
        kh, ks = G.condition_numbers(p, a_run) if p.kind != 3 else (None, None)
        us = {"fp64": 1.11e-16, "fp32": 5.96e-8, "bf16": 3.91e-3}[pn]
        x.zero_()
        H.solve(b, x, a_run, omega, prec, TOL, min(3, mit), tol_h=tin, tol_s=tin)  # warm-up
        x.zero_()
        st, s = H.solve(b, x, a_run, omega, prec, TOL, mit, tol_h=tin, tol_s=tin,
                        alpha_restarts=args.alpha_restarts)
        H.apply(G.OP_A, x, r)
        relres = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
        ab = algorithmic_bytes(p.npoints, s, sbytes, dbytes)
        ach = ab / s["seconds"] / 1e9
        print(json.dumps({
            "metric": "time to 1e-10 rel. backward error: mixed vs FP64 GADI, 1 GB300; HBM %peak",
            "workload": name, "config": {"workload": desc, "alpha": a_run, "alpha_over_alpha_star":
                                          a_run / alpha_star(p), "omega": omega, "u_s": pn,
                                          "tol_inner": tin, "maxit": mit, "alpha_select": bool(args.alpha_select),
                                          "alpha_restarts": args.alpha_restarts},
            "eq_4_1": {"kappa_h": kh, "kappa_s": ks, "kappa_h_kappa_s_u_s": kh * ks * us if kh else None,
                       "tau": args.tau},
            "alpha_final": s["alpha"], "restarts": s["restarts"],
            "value": s["seconds"], "unit": "s", "status": G.status_str(st), "outer_its": s["outer_its"],
            "inner_its_h": s["inner_its_h"], "inner_its_s": s["inner_its_s"], "relres": relres,
            "ms_per_outer": 1e3 * s["seconds"] / max(1, s["outer_its"]),
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "peak_source": src}}), flush=True)


def run_phases(args):
    """Each step of Algorithm 1 on its own, through the single-step entry
    points (one launch each), on the 3D workload at --grid3 (or the 2D one at
    --grid with --phase-grid 2d): the residual step (x + y, b - A x, ||r||,
    r_s), CG on H and CGNR on S with a fixed iteration count.  The time of
    one inner iteration is the difference of two counts (20 and 10) over 10,
    which removes launch and set-up.  One JSON line per (precision, phase) with
    the algorithmic bytes (residual 3d + 2s, CG / CGNR iteration 8s per
    point) per second against the HBM peak."""
    import torch

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import alpha_star, config2, config3
    B.build()
    if args.phase_grid == "2d":
        p, xt = config2(args.grid)
        wl = f"conv-diff-2d {args.grid}^2"
    else:
        p, xt = config3(args.grid3)
        wl = f"conv-diff-3d {args.grid3}^3"
    n = p.npoints
    hbm, src = _peaks()
    H = G.Gadi.from_problem(p)
    xtd = torch.from_numpy(xt).cuda()
    b = torch.zeros_like(xtd)
    H.apply(G.OP_A, xtd, b)
    x = (xtd * 0.5).contiguous()
    xo = torch.empty_like(x)
    alpha = args.alpha_factor * alpha_star(p)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record(stream)
            fn()
            ev1.record(stream)
            torch.cuda.synchronize()
            ts.append(ev0.elapsed_time(ev1) / 1e3)
        return statistics.median(ts)

    for pn in args.precs.split(","):
        prec = {"fp64": G.FP64, "fp32": G.FP32, "bf16": G.BF16}[pn]
        sb = {"fp64": 8, "fp32": 4, "bf16": 2}[pn]
        dt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.int16}[pn]
        y = torch.zeros(n, dtype=dt, device="cuda")
        rs = torch.empty(n, dtype=dt, device="cuda")
        z = torch.empty(n, dtype=dt, device="cuda")
        yv = torch.empty(n, dtype=dt, device="cuda")
        H.step_residual(prec, b, x, y, xo, None, rs)  # warm-up; rs = the right-hand side below
        t_res = timed(lambda: H.step_residual(prec, b, x, y, xo, None, rs))
        lines = [("residual", t_res, 1, (3 * 8 + 2 * sb) * n)]
        H.step_solve_h(alpha, prec, rs, z, 0.0, 2)
        ih = {k: H.step_solve_h(alpha, prec, rs, z, 0.0, k) for k in (10, 20)}
        th = {k: timed(lambda k=k: H.step_solve_h(alpha, prec, rs, z, 0.0, k)) for k in (10, 20)}
        lines.append(("cg_h", (th[20] - th[10]) / max(1, ih[20] - ih[10]), ih, 8 * sb * n))
        H.step_solve_s(alpha, OMEGA, prec, z, yv, 0.0, 2, 0, False)
        is_ = {k: H.step_solve_s(alpha, OMEGA, prec, z, yv, 0.0, k, 0, False) for k in (10, 20)}
        ts_ = {k: timed(lambda k=k: H.step_solve_s(alpha, OMEGA, prec, z, yv, 0.0, k, 0, False)) for k in (10, 20)}
        lines.append(("cgnr_s", (ts_[20] - ts_[10]) / max(1, is_[20] - is_[10]), is_, 8 * sb * n))
        for name, t, its, ab in lines:
            print(json.dumps({"metric": "per-step device time and algorithmic bandwidth", "workload": wl,
                              "phase": name, "u_s": pn, "ms": t * 1e3, "alg_bytes": ab,
                              "GBps": ab / t / 1e9, "frac": ab / t / 1e9 / hbm, "peak": hbm,
                              "iterations": its if isinstance(its, dict) else None,
                              "peak_source": src,
                              "note": "inner phases: per iteration (difference of 20 and 10 iterations)"}),
                  flush=True)
    H.close()


def run_csr(args):
    """The headline workload's matrix (2048^2 2D convection-diffusion, beta
    by seed 2) assembled as CSR and solved by the CSR kernels (the paper's own
    storage, Sec. 5.1), FP32 inner, alpha = 8 alpha*, omega = 0, beside the
    stencil kernels on the same system.  Reported: time to 1e-10, iterations
    and the bytes the CSR path moves per solve (vectors as for the stencil,
    plus the matrices: each SpMV reads its values in u_s (A in FP64), column
    indices and row pointers)."""
    import torch

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import K_CSR, Problem, alpha_star, config2
    B.build()
    p, xt = config2(args.grid)
    rp, cl, vl = G.stencil_csr(p)
    pc = Problem(K_CSR, p.npoints, rowptr=rp, col=cl, val=vl)
    t0 = time.perf_counter()
    Hc = G.Gadi.from_problem(pc)
    t_create = time.perf_counter() - t0
    Hs = G.Gadi.from_problem(p)
    xtd = torch.from_numpy(xt).cuda()
    b = torch.zeros_like(xtd)
    Hs.apply(G.OP_A, xtd, b)
    x = torch.zeros_like(b)
    alpha = ALPHA_FACTOR * alpha_star(p)
    hbm, src = _peaks()
    n, nnz_a = p.npoints, len(vl)
    nnz_m = nnz_a  # M and N share A's pattern here (symmetric pattern, full diagonal)
    for name, H in (("csr", Hc), ("stencil", Hs)):
        x.zero_()
        H.solve(b, x, alpha, OMEGA, G.FP32, TOL, 3, tol_h=TOL_H, tol_s=TOL_S)  # warm-up
        x.zero_()
        st, s_ = H.solve(b, x, alpha, OMEGA, G.FP32, TOL, args.maxit, tol_h=TOL_H, tol_s=TOL_S)
        r = torch.zeros_like(b)
        Hs.apply(G.OP_A, x, r)
        relres = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
        vec = algorithmic_bytes(n, s_, 4)
        mat = 0.0
        if name == "csr":
            # per SpMV: values + column indices (+ row pointers); A in FP64
            spmv_us = nnz_m * (4 + 4) + 4 * (n + 1)
            spmv_a = nnz_a * (8 + 4) + 4 * (n + 1)
            k = s_["outer_its"]
            mat = (k + 1) * spmv_a + spmv_us * (s_["inner_its_h"] + 2 * s_["inner_its_s"] + k)
        print(json.dumps({
            "metric": "time to 1e-10 relative residual, CSR kernels vs stencil kernels", "workload": "csr2d",
            "kernels": name, "config": {"workload": WORKLOAD + " assembled as CSR" if name == "csr" else WORKLOAD,
                                        "alpha_over_alpha_star": ALPHA_FACTOR, "omega": OMEGA, "u_s": "fp32",
                                        "nnz": nnz_a if name == "csr" else None},
            "value": s_["seconds"], "unit": "s", "status": G.status_str(st), "outer_its": s_["outer_its"],
            "inner_its_h": s_["inner_its_h"], "inner_its_s": s_["inner_its_s"], "relres": relres,
            "bytes": vec + mat, "GBps": (vec + mat) / s_["seconds"] / 1e9,
            "frac": (vec + mat) / s_["seconds"] / 1e9 / hbm, "peak": hbm, "peak_source": src,
            "create_s": t_create if name == "csr" else None}), flush=True)
    Hc.close()
    Hs.close()


def run_batched(args):
    """Config 5: 96 uneven 2D systems x 4 right-hand sides in one persistent
    launch (FP32 inner, FP64 outer), literal alpha ~ logU[1e-2,10] capped at
    --maxit5 outer iterations per unit, and a batch with alpha = alpha*(N) x
    logU[0.5,2].  Reports solves/s (converged units per second of the launch),
    the converged fraction and p50/p99 of the per-unit device times."""
    import numpy as np
    import torch

    import paper_2512_21164_gb300 as G
    from paper_2512_21164_gb300 import build as B
    from workloads import config5
    B.build()
    for scaled in (False, True):
        systems = config5(args.nsys5, 4, scaled_alpha=scaled)
        hs, bs, xs, al = [], [], [], []
        for p, a, xts in systems:
            H = G.Gadi.from_problem(p)
            xt = torch.from_numpy(np.concatenate(xts)).cuda()
            b = torch.zeros_like(xt)
            for j in range(4):
                H.apply(G.OP_A, xt[j * p.nvec:(j + 1) * p.nvec], b[j * p.nvec:(j + 1) * p.nvec])
            hs.append(H)
            bs.append(b)
            xs.append(torch.zeros_like(b))
            al.append(a)
        maxit = args.maxit5 if not scaled else 20000
        tune_s = None
        hres = {} if args.hres5 < 0 else {"h_resident": args.hres5}
        if args.group5 <= 0:
            # the group-size tuner runs on the first batch of these grids and
            # alpha values in the process (timed here, outside the measured
            # launch); a 2-iteration batch triggers it
            xw = [torch.zeros_like(v) for v in xs]
            t0 = time.perf_counter()
            G.solve_batched(hs, 4, bs, xw, al, OMEGA, G.FP32, TOL, 2, tol_h=TOL_INNER, tol_s=TOL_INNER,
                            batch_group=args.group5, batch_interleave=args.interleave5, **hres)
            tune_s = time.perf_counter() - t0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        st, stats = G.solve_batched(hs, 4, bs, xs, al, OMEGA, G.FP32, TOL, maxit, batch_interleave=args.interleave5, **hres,
                                    tol_h=TOL_INNER,
                                    tol_s=TOL_INNER, batch_group=args.group5)
        ev1.record()
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        conv = [u for u in stats if u["status"] == G.OK]
        t = np.array([u["seconds"] for u in conv]) if conv else np.array([0.0])
        print(json.dumps({
            "metric": "batched GADI solves/s (time to 1e-10 per unit)", "workload": "c5",
            "config": {"workload": f"{len(systems)} 2D conv-diff systems N in {{128,256,512,1024}}, 4 rhs each",
                       "alpha": "alpha*(N) x logU[0.5,2]" if scaled else "logU[1e-2,10]", "omega": OMEGA,
                       "maxit": maxit, "u_s": "fp32", "batch_group": args.group5,
                       "interleaved_rhs": bool(args.interleave5),
                       "h_solve": "p in shared memory" if stats[0]["h_resident"] else "streaming"},
            "group_blocks": {f"N={n}": {str(k): int(v) for k, v in zip(*np.unique(
                [u["blocks"] for i, u in enumerate(stats) if systems[i // 4][0].nx == n], return_counts=True))}
                for n in sorted({sp.nx for sp, _, _ in systems})},
            "per_class": {f"N={n}": {
                "p50_s": float(np.median([u["seconds"] for i, u in enumerate(stats) if systems[i // 4][0].nx == n])),
                "max_s": float(np.max([u["seconds"] for i, u in enumerate(stats) if systems[i // 4][0].nx == n])),
                "outer_p50": float(np.median([u["outer_its"] for i, u in enumerate(stats)
                                              if systems[i // 4][0].nx == n])),
                "units": int(sum(1 for i in range(len(stats)) if systems[i // 4][0].nx == n))}
                for n in sorted({sp.nx for sp, _, _ in systems})},
            "tune_s": tune_s,
            "value": len(conv) / sec, "unit": "solves/s", "seconds": sec, "units": len(stats),
            "converged": len(conv), "p50_s": float(np.percentile(t, 50)), "p99_s": float(np.percentile(t, 99)),
            "status": G.status_str(st)}), flush=True)
        for H in hs:
            H.close()


TWIN = 256  # the CPU oracle's twin of the 2048^2 workload (same beta draw, alpha/alpha*, omega, tolerances)


def _twin():
    from workloads import SEED_C2, alpha_star, conv_diff_2d
    p, xt = conv_diff_2d(TWIN, SEED_C2)
    return p, xt, ALPHA_FACTOR * alpha_star(p)


def _twin_desc():
    return (f"conv-diff-2d {TWIN}x{TWIN} twin of the {WORKLOAD} workload (same beta draw, alpha = "
            f"{ALPHA_FACTOR:g} alpha* of the twin, omega = {OMEGA:g}, tol_h = tol_s = {TOL_H:g}, FP32 inner), "
            f"solved to 1e-10 by the C oracle")


def _oracle_solve(omp, p, xt, alpha):
    """One oracle solve of Algorithm 1 to 1e-10 (FP64 outer, FP32 inner);
    returns (seconds, stats)."""
    import oracle as O
    orc = O.Oracle(p, omp=omp)
    b = orc.rhs(xt)
    t0 = time.perf_counter()
    _, st = orc.gadi(b, alpha, OMEGA, O.FP32, tol=TOL, maxit=MAXIT, tol_h=TOL_H, tol_s=TOL_S)
    return time.perf_counter() - t0, st


def _omp_threads():
    return int(os.environ.get("OMP_NUM_THREADS", "0")) or (os.cpu_count() or 1)


def cpu_baseline():
    """The CPU oracle timed to tolerance on this host (no extrapolation):
    the 256^2 twin of the workload single-threaded (the oracle as it stands,
    the reported value) and in the all-core OpenMP build, and config 1
    (64^2, plain FP64, alpha 0.5, omega 1, 500-iteration cap) at full size."""
    import oracle as O
    from workloads import config1
    p, xt, alpha = _twin()
    t1, st1 = _oracle_solve(False, p, xt, alpha)
    out = {"value": t1, "unit": "s", "cores": 1, "kind": "oracle",
           "sample": _twin_desc() + f", single thread: {st1['status']} after {st1['outer_its']} outer / "
                     f"{st1['inner_h']} H / {st1['inner_s']} S iterations, relres {st1['relres']:.3g}",
           "host_cpus": os.cpu_count()}
    if O.has_openmp():
        tm, stm = _oracle_solve(True, p, xt, alpha)
        out["openmp"] = {"value": tm, "unit": "s", "cores": _omp_threads(), "status": stm["status"],
                         "outer_its": stm["outer_its"]}
    else:
        out["openmp"] = {"unavailable": "gcc without OpenMP on this host"}
    p1, xt1, c = config1()
    orc = O.Oracle(p1)
    b1 = orc.rhs(xt1)
    t0 = time.perf_counter()
    _, s1 = orc.gadi(b1, c["alpha"], c["omega"], O.FP64, tol=c["tol"], maxit=c["maxit"])
    out["config1"] = {"value": time.perf_counter() - t0, "unit": "s", "cores": 1, "status": s1["status"],
                      "outer_its": s1["outer_its"], "relres": s1["relres"],
                      "workload": "conv-diff-2d 64x64, beta=(10,10), alpha=0.5, omega=1, maxit 500, plain FP64"}
    return out


def run_reference(args):
    """The CPU oracle (all-core OpenMP build where gcc has OpenMP, else the
    single-threaded one) solving the 256^2 twin of the workload to 1e-10,
    once per step: a real bounded run, timed on the host cores, rank 0 only."""
    import oracle as O
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    omp = O.has_openmp()
    p, xt, alpha = _twin()
    vals, st = [], None
    for i in range(args.warmup + args.steps):
        dt, st = _oracle_solve(omp, p, xt, alpha)
        if i >= args.warmup:
            vals.append(dt)
    v = statistics.mean(vals)
    cores = _omp_threads() if omp else 1
    cb = {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
          "sample": _twin_desc() + f" ({'OpenMP, all host cores' if omp else 'single thread'}): "
                    f"{st['status']} after {st['outer_its']} outer iterations, relres {st['relres']:.3g}"}
    out = {"metric": "time to 1e-10 rel. backward error: mixed vs FP64 GADI, 1 GB300; HBM %peak",
           "value": v, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 outer / f32 inner", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"conv-diff-2d {TWIN}x{TWIN} (twin of the 2048x2048 workload)",
                      "twin_of": WORKLOAD, "alpha_over_alpha_star": ALPHA_FACTOR, "omega": OMEGA,
                      "tol_h": TOL_H, "tol_s": TOL_S, "u_s": "fp32", "u": "fp64"},
           "step_s": vals, "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=2048)
    ap.add_argument("--maxit", type=int, default=MAXIT)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-case", choices=["fp64", "fp32", "bf16"], default=None,
                    help="run one solve capped at --maxit outer iterations (for ncu) and exit")
    ap.add_argument("--grids", default=None, help="paper2d / paper3d / paperc: comma-separated grid sizes")
    ap.add_argument("--precs", default="fp64,fp32,bf16", help="inner precisions to run (paper*, c1, c3, c4, phases)")
    ap.add_argument("--alpha-factors", default=None,
                    help="paper2d / paper3d / paperc: alpha/alpha*:omega pairs tried, or gpr[:omega] for the "
                         "alpha of a GPR trained on small instances (Sec. 4.2)")
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c1", "c3", "c4", "c5", "c2dd", "paper2d", "paper3d", "paperc", "phases", "csr2d", "c2s"],
                    help="c2 (default): the headline line; others: per-precision lines")
    ap.add_argument("--grid3", type=int, default=512)
    ap.add_argument("--phase-grid", choices=["2d", "3d"], default="3d", help="phases: the 2D or the 3D workload")
    ap.add_argument("--grid4", type=int, default=4096)
    ap.add_argument("--alpha-factor", type=float, default=4.0)
    ap.add_argument("--alpha-select", action="store_true",
                    help="c3/c4: start from the alpha of Sec. 4.3's condition check (gadi_select_alpha)")
    ap.add_argument("--alpha-restarts", type=int, default=0, help="c3/c4: Sec. 4.3 restarts with 2 alpha")
    ap.add_argument("--tau", type=float, default=0.01)
    ap.add_argument("--omega", type=float, default=None, help="c3: omega (default that of the 2048^2 line)")
    ap.add_argument("--fp64-maxit", type=int, default=20000)
    ap.add_argument("--maxit5", type=int, default=2000)
    ap.add_argument("--nsys5", type=int, default=96)
    ap.add_argument("--interleave5", type=int, default=0, help="c5: 1 = the four right-hand sides of a system in one unit")
    ap.add_argument("--group5", type=int, default=0, help="c5: blocks per group (0 = the library's tuner)")
    ap.add_argument("--hres5", type=int, default=-1,
                    help="c5: 0 = units take the streaming H-solve (default: the library's, p in shared memory)")
    ap.add_argument("--record-traffic", nargs=2, metavar=("NCU_REPORT", "PROFILE_CASE_LOG"), default=None,
                    help="write the committed traffic record from an ncu report of --profile-case")
    args = ap.parse_args()
    if args.record_traffic:
        record_traffic(*args.record_traffic)
    elif args.profile_case:
        run_profile_case(args)
    elif args.workload == "c5" and args.impl == "ours":
        run_batched(args)
    elif args.workload == "phases" and args.impl == "ours":
        run_phases(args)
    elif args.workload == "csr2d" and args.impl == "ours":
        run_csr(args)
    elif args.workload == "c2dd" and args.impl == "ours":
        run_c2_dd(args)
    elif args.workload in ("paper2d", "paper3d", "paperc") and args.impl == "ours":
        run_paper(args)
    elif args.workload != "c2" and args.impl == "ours":
        run_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
