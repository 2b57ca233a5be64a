#!/usr/bin/env python
"""Benchmark: s-step PCG solve time and HBM GB/s vs plain PCG on one GB300.

Workload (default): 3-D Poisson, 7-point stencil on a 256^3 grid
(n = 16,777,216, nnz = 117,047,296), CSR FP64 input, Jacobi, s = 4 monomial
basis, x_true ~ U[-1, 1) from seed 0, b = A x_true, x0 = 0, stop at
recursive rel. residual 1e-8.  One step = one complete solve (init, every
outer step, export of x, true residual) through the C ABI.

Reported:
  value      whole-job bandwidth of the s-step solves: the bytes the solve's
             kernels move (the per-kernel byte model below) over the solve's
             device time, summed over ranks; it cannot exceed the copy
             bandwidth.  value_yardstick_gbs divides the bytes Algorithm 3 moves
             on the system as given (CSR with FP64 values, FP64 vectors, A U and
             A P stored: the yardstick below) by the same time.
  dtype      the arithmetic of the solve: f64 (default) or df64 (pairs of FP32)
  e2e        the same metric through the public API with host buffers
             (b, x0 copied in and x copied out inside the timed region)
  roofline   the dominant kernel family, timed by the library's CUDA events
             on its own stream over the timed steps.  In FP64 the kernels are
             bound by the FP64 units (about 2 operations per clock per SM on a
             GB300, 1/60 of the FP32 rate): "alu", FP64 operations per launch
             (fp64_ops_model) over the launch's duration against 2 per clock
             per SM at the maximum SM clock; in df64 "hbm", the bytes the
             kernels move against the measured copy bandwidth
  pcg_*      plain PCG (Algorithm 1) on the same kernels and arithmetic
  pfcg_*     PFCG-NN (Algorithm 2, one reduction per iteration), likewise
  df64_*     (FP64 runs) the same solve and PCG in double-float
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same solve

Yardstick (bytes per solve, V = 8 n, M = 12 nnz + 4 (n+1)): init M + 5V,
final M + 2V, per outer step s levels of M + 2V (+ 2V when j < s-1) and the
block update (6s + 6) V ((4s + 6) V in the first step); PCG per iteration
M + 13V.

Per-kernel byte model (bytes per launch; V = 8 n, M = 4 (n+1) + nnz (4 + value bytes)):
  MPK level j     M + 3V: u_j gathered, 1/diag read, u_{j+1} = D^-1 A u_j
                  written (A u_j is not stored)
  block update    (5s + 5) V: U_1..U_{s+1}, P_old, Q_old, x, diag read;
                  P, Q, x and the next z written (first step: (2s + 5) V)
  A matrix in the constant-coefficient diagonal form (the 7-point stencil)
  replaces M by 4n (one presence mask per row) in the levels and PCG's SpMV,
  and reads no 1/diag or diag vector: level 4n + 2V, update (5s + 4) V.
  (with --fused-mpk the levels and update of the A U / A P form are timed:
  levels M + 2V, + 2V when j < s-1; update (6s + 6) V, first (4s + 6) V)
  init            M + 5V: x0 gathered, b, 1/diag read, r, z written
                  (DF64: + V, the zeroed correction)
  final           M + 2V: x gathered, b read (DF64: + 3V, x = x0 + correction)
PCG per iteration: SpMV + p.Ap M + 2V; update 7V; direction 4V (diagonal
form: 4n + 2V, 6V, 3V).

Multi-GPU: replicas only.  Every rank solves its own system (seed = rank)
with no collective on the data path; value = all ranks' bytes / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s-step PCG solve time & HBM GB/s vs plain PCG, 1×GB300, rel. residual 1e-8"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="sscg", choices=["sscg", "reference"])
    p.add_argument("--N", type=int, default=256)
    p.add_argument("--s", type=int, default=4)
    p.add_argument("--arith", default="f64", choices=["f64", "df64"])
    p.add_argument("--no-df64", action="store_true", help="skip the double-float solve and PCG beside the FP64 line")
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--no-pcg", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="skip the s in {1,2,4,6,8} sweep")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--fused-mpk", action="store_true", help="several matrix-powers levels per launch (L2-resident)")
    p.add_argument("--fma-update", action="store_true",
                   help="FP64, s <= 4: form the block update's P and Q with FP64 FMAs instead of fixed point")
    p.add_argument("--workload", default="poisson", choices=["poisson", "batch", "mixed27", "cheb", "peaks"],
                   help="poisson: one 7-point solve (the headline); batch: the batched serving mix; "
                        "mixed27: 27-point 192^3 in mixed precision to 1e-10; cheb: Chebyshev basis with "
                        "network vs Lanczos intervals on variable-coefficient 128^3 fields; peaks: the "
                        "arithmetic throughput probes (FP64 FMA/add/multiply, FP64 mma, FP32 FMA, integer)")
    p.add_argument("--batch-systems", type=int, default=64)
    p.add_argument("--batch-nmin", type=int, default=32, help="batch: smallest grid edge of the mix")
    p.add_argument("--batch-nmax", type=int, default=160, help="batch: largest grid edge of the mix")
    p.add_argument("--no-tune", action="store_true", help="batch: fixed tiles instead of the autotuner")
    p.add_argument("--no-seq", action="store_true", help="batch: skip the one-at-a-time comparison")
    p.add_argument("--persistent", action="store_true", help="batch: one cooperative launch per solve")
    return p.parse_args()


# ------------------------------------------------------------ byte model

# DRAM bytes (read + write) per row and launch that ncu --set full measured
# for this workload's kernels (7-point stencil in the diagonal form, s = 4,
# sequential levels) at n = 4,096,000: a level (mean of the captured
# launches; at that size L2 still holds most of the level's writes when it
# ends) and the block update, per arithmetic and update kernel (profiles/
# k_update_fix_k_level_poisson7_160_f64_s4.txt, k_level_k_update_q_poisson7_160_f64_s4.txt,
# k_level_dia_k_update_q_poisson7_160_df64_s4.txt).
# The roofline's "traffic" scales them to the workload's n; it is null for any
# other configuration.
L2_BYTES = 129 * 10 ** 6  # the GB300's L2
L2_FLUSH_BYTES = 256 << 20

NCU_TRAFFIC_PER_ROW = {
    "f64": {"mpk": 53.86e6 / 4.096e6, "update": 734.1e6 / 4.096e6},
    "f64-fixed": {"update": 733.296e6 / 4.096e6},
    "df64": {"mpk": 54.0e6 / 4.096e6, "update": 732.694e6 / 4.096e6},
}


def byte_model(n, nnz, vbytes, s, arith, fused=False, dia=False):
    V = 8 * n
    M = 4 * (n + 1) + nnz * (4 + vbytes)
    df = arith != "f64"
    # diagonal form: a 4-byte mask per row replaces the CSR arrays in the
    # levels and PCG's SpMV, and the constant diagonal replaces 1/diag reads
    Md, dv = (4 * n, 0) if dia else (M, V)
    if fused:
        lv = [M + 2 * V + (2 * V if j < s - 1 else 0) for j in range(s)]
        upd, upd_first = (6 * s + 6) * V, (4 * s + 6) * V
    else:
        lv = [Md + 2 * V + dv for j in range(s)]
        upd, upd_first = (5 * s + 4) * V + dv, (2 * s + 4) * V + dv
    return dict(M=M, V=V, level=lv, level_avg=sum(lv) / s, update=upd, update_first=upd_first,
                init=M + 5 * V + (V if df else 0), final=M + 2 * V + (3 * V if df else 0),
                pcg_spmv=Md + 2 * V, pcg_update=6 * V + dv, pcg_dir=3 * V + dv)


def traffic(a, family, n, dia, fixed=False):
    """Measured DRAM bytes per launch of `family`, scaled to n rows, or None."""
    per = NCU_TRAFFIC_PER_ROW.get(a.arith + ("-fixed" if fixed and family == "update" else ""))
    if per is None or a.s != 4 or a.fused_mpk or not dia or family not in per:
        return None
    return round(per[family] * n)


def yardstick(n, nnz, s):
    """The fixed model behind `value` (see the module docstring)."""
    return byte_model(n, nnz, 8, s, "f64", fused=True, dia=False)


def sstep_bytes(bm, outer):
    if outer == 0:
        return bm["init"] + bm["final"]
    return (bm["init"] + bm["final"] + outer * sum(bm["level"]) + bm["update_first"]
            + (outer - 1) * bm["update"])


def pcg_bytes(bm, iters):
    return bm["init"] + bm["final"] + iters * (bm["pcg_spmv"] + bm["pcg_update"] + bm["pcg_dir"])


# ---------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ distributed

def dist_setup(gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v):
    if pg is None:
        return v
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v):
    if pg is None:
        return v
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------- CPU (oracle)

def oracle_sample(sysm, s, budget_s, tol):
    """Time the oracle's s-step solve on a bounded number of outer steps."""
    import oracle

    M = oracle.as_matrix(sysm)
    t0 = time.perf_counter()
    oracle.pcgs(M, sysm["b"], s, tol=0.0, maxit=1)
    one = time.perf_counter() - t0
    steps = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    r = oracle.pcgs(M, sysm["b"], s, tol=0.0, maxit=steps)
    dt = time.perf_counter() - t0
    return dict(steps=r.iters, seconds=dt, threads=oracle.num_threads())


def hbm_peak():
    """The measured copy bandwidth (MEASURED_PEAKS.json), else the fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), \
            "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def family_roofline(res, bytes_per_record, names):
    """Roofline of a solve's dominant kernel family from the library's CUDA
    events (profile=True): bytes_per_record[f] are the algorithmic bytes of one
    timed record of family f, names[f] its kernels."""
    fam = {}
    for f in bytes_per_record:
        t, c = res.profile[f"t_{f}_ms"], res.profile[f"n_{f}"]
        if c:
            fam[f] = (t, c)
    dom = max(fam, key=lambda f: fam[f][0])
    t, c = fam[dom]
    achieved = bytes_per_record[dom] / (t / c * 1e-3) / 1e9
    peak, src = hbm_peak()
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "kernel": names[dom], "peak_source": src,
            "family_ms_per_solve": {f: round(v[0], 3) for f, v in fam.items()}}


def family_alu_roofline(res, ops_per_record, names, sm_count):
    """FP64 ALU roofline of a solve's dominant kernel family from the library's
    CUDA events: ops_per_record[f] FP64 operations per timed record of f."""
    fam = {}
    for f in ops_per_record:
        t, c = res.profile[f"t_{f}_ms"], res.profile[f"n_{f}"]
        if c:
            fam[f] = (t, c)
    dom = max(fam, key=lambda f: fam[f][0])
    t, c = fam[dom]
    peak = alu_peak(sm_count)
    achieved = ops_per_record[dom] / (t / c * 1e-3)
    return {"bound": "alu", "achieved": round(achieved / 1e9, 1), "peak": round(peak / 1e9, 1), "unit": "Gop/s",
            "frac": round(achieved / peak, 4), "traffic": None, "kernel": names[dom],
            "peak_source": "FP64 operations at 2 per clock per SM x SMs x 2070 MHz (nominal 1.25 TFLOP/s)",
            "family_ms_per_solve": {f: round(v[0], 3) for f, v in fam.items()},
            "family_frac": {f: round(ops_per_record[f] / (v[0] / v[1] * 1e-3) / peak, 4) for f, v in fam.items()}}


def workload_name(N, s, arith):
    n = N ** 3
    return (f"poisson7 {N}^3 (n={n:,}), CSR FP64 input, Jacobi, s={s} monomial, b=A x_true, x_true~U[-1,1) "
            f"seed=rank, x0=0, tol 1e-8; arithmetic {arith}")


def fp64_ops_model(s, K=7, fixed_update=False):
    """FP64-pipe operations per row of the FP64 kernels on a Laplacian-class
    stencil in the diagonal form under a constant Jacobi scale.  One DFMA,
    DADD or DMUL per thread is one operation, and so is each conversion of a
    64-bit fixed-point sum to FP64: a GB300 issues that conversion to the FP64
    pipe at its rate (the I2F64 probe of include/sscg_probe.h).  The neighbour
    sum itself runs on the integer units (csrc/fixsum.cuh), whatever K, and
    costs one conversion.  Level j: the conversion, one FMA for u_{j+1} and one
    for each moment (the second moment is skipped on the last level); block
    update: s^2 FMAs each for P and Q (with the fixed-point update none: P and
    Q are integer dot products, one conversion each), s FMAs each for x and z,
    one for sum z^2 (first step: no P, Q); PCG: SpMV the conversion, one FMA
    for A p and one for p . Ap; update x, r, ||r||^2; direction u = D^-1 r and
    p = u + beta p."""
    lvl = [3 + (1 if 2 * j + 2 <= 2 * s - 1 else 0) for j in range(s)]
    upd = 4 * s + 1 if fixed_update else 2 * s * s + 2 * s + 1
    return dict(level=lvl, level_avg=sum(lvl) / s, update=upd, update_first=2 * s + 1,
                pcg_spmv=3, pcg_update=3, pcg_dir=2)


def fixed_update_used(a):
    """The FP64 block update forms P and Q in fixed point at s <= 6 (csrc/kernels.cuh k_update_fix)."""
    return a.arith == "f64" and a.s <= 6 and not a.fma_update and not a.fused_mpk


def alu_peak(sm_count, mhz=2070.0):
    """The FP64 ALU roof in operations per second: 2 FP64 operations per clock
    per SM (the nominal 1.25 TFLOP/s of a GB300 at its 2070 MHz maximum SM
    clock is 1.25e12 / 2 / 152 / 2.07e9 = 1.99 FMAs per clock per SM)."""
    return fp64_alu_peak(sm_count, mhz)


def main():
    a = parse()
    world, rank, local, pg = dist_setup(a.gpus)
    from paper_2501_03743_gb300 import inputs

    if a.impl == "reference":
        return reference_arm(a, world, rank, pg)
    if a.workload == "batch":
        return run_batch(a, world, rank, local, pg)
    if a.workload == "mixed27":
        return run_mixed27(a, world, rank, local, pg)
    if a.workload == "cheb":
        return run_cheb(a, world, rank, local, pg)
    if a.workload == "peaks":
        return run_peaks(a, world, rank, local, pg)

    import torch

    if rank == 0:
        from paper_2501_03743_gb300 import build

        build.build()
    barrier(pg)
    torch.cuda.set_device(local)
    from paper_2501_03743_gb300 import sscg

    sysm = inputs.system("poisson7", a.N, seed=rank)
    n, nnz = sysm["n"], len(sysm["col"])
    ctx = sscg.Context()
    A = sscg.Matrix(ctx, sysm["rowptr"], sysm["col"], sysm["val"])
    props = A.props()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count

    def model(arith):
        vbytes = 8 if arith == "f64" else (4 if props["values_exact_fp32"] else 8)
        dia = props["format"] == 1 and not a.fused_mpk
        return byte_model(n, nnz, vbytes, a.s, arith, fused=a.fused_mpk, dia=dia), dia

    bm, dia = model(a.arith)
    ym = yardstick(n, nnz, a.s)
    b = torch.from_numpy(sysm["b"]).cuda()
    x = torch.zeros_like(b)
    # the timed solves record no per-kernel events; a profiled solver of the same
    # solve, run after the timed region, gives the kernel families' times
    solver = sscg.Solver(A, s=a.s, tol=a.tol, maxit=5000, arith=a.arith,
                         fused_mpk=a.fused_mpk, fma_update=a.fma_update)
    stream = ctx.stream

    def timed(fn, count):
        evs = []
        out = []
        for _ in range(count):
            x.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out.append(fn())
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in evs], out

    for _ in range(a.warmup):
        x.zero_()
        solver.solve(b, x)
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                    if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    ms, res = timed(lambda: solver.solve(b, x), a.steps)
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(pg)
    r0 = res[-1]
    total_ms = max_over_ranks(pg, sum(ms))
    ms_per_step = total_ms / a.steps
    yard_solve = sstep_bytes(ym, r0.outer_iters)
    kernel_bytes_solve = sstep_bytes(bm, r0.outer_iters)
    # value: the bytes the solve's kernels move (their algorithmic byte model) per second
    value = sum_over_ranks(pg, kernel_bytes_solve * a.steps) / (total_ms * 1e-3) / 1e9
    value_yard = sum_over_ranks(pg, yard_solve * a.steps) / (total_ms * 1e-3) / 1e9

    # kernel families: the library's CUDA events on its stream, over profiled runs
    # of the same solve (the events between kernels stay out of the timed region)
    prof_solver = sscg.Solver(A, s=a.s, tol=a.tol, maxit=5000, arith=a.arith, profile=True,
                              fused_mpk=a.fused_mpk, fma_update=a.fma_update)
    _, pres_s = timed(lambda: prof_solver.solve(b, x), max(1, min(a.steps, 3)))
    nprof = len(pres_s)
    del prof_solver
    fixed = fixed_update_used(a)
    ops = fp64_ops_model(a.s, fixed_update=fixed)
    fam = {}
    for key, cnt, per, fops in (("mpk", "n_mpk", bm["level_avg"], ops["level_avg"]),
                                ("update", "n_update", bm["update"], ops["update"])):
        t = sum(r.profile[f"t_{key}_ms"] for r in pres_s)
        c = sum(r.profile[cnt] for r in pres_s)
        fam[key] = dict(ms=t, launches=c, bytes_per_launch=per, ops_per_launch=fops * n)
    dom = max(fam, key=lambda k: fam[k]["ms"])
    d = fam[dom]
    avg_s = d["ms"] / max(d["launches"], 1) * 1e-3
    hbm, hbm_src = hbm_peak()
    kernel_names = {"mpk": ("k_level (matrix-powers level: diagonal-form SpMV + Jacobi + moments)" if dia else
                            "k_level (matrix-powers level: CSR SpMV + Jacobi + moments)"),
                    "update": ("k_update_tma (block update P, AP, x, r + next z)" if a.fused_mpk else
                               "k_update_fix (block update: P, Q = D^-1 A P as fixed-point dot products on the "
                               "integer multipliers; x, z FP64 FMAs)" if fixed else
                               "k_update_q (block update P, Q = D^-1 A P, x, z)")}
    gbs = {k: round(v["bytes_per_launch"] / (v["ms"] / max(v["launches"], 1) * 1e-3) / 1e9, 1) for k, v in fam.items()}
    if a.arith == "f64" and dia and not a.fused_mpk:
        peak = alu_peak(sm_count)
        gops = {k: round(v["ops_per_launch"] / (v["ms"] / max(v["launches"], 1) * 1e-3) / 1e9, 1)
                for k, v in fam.items()}
        achieved = d["ops_per_launch"] / avg_s / 1e9
        fp64_frac = achieved * 1e9 / peak
        hbm_frac = gbs[dom] / hbm
        if fp64_frac >= hbm_frac:  # the dominant kernel's binding roof: the larger of its two fractions
            head = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak / 1e9, 1), "unit": "Gop/s",
                    "frac": round(fp64_frac, 4),
                    "peak_source": f"FP64 operations (DFMA/DADD/DMUL per thread) at 2 per clock per SM x "
                                   f"{sm_count} SMs x 2070 MHz, from the nominal 1.25 TFLOP/s and maximum SM clock; "
                                   "the probe of include/sscg_probe.h measures 529 Gop/s"}
        else:
            head = {"bound": "hbm", "achieved": gbs[dom], "peak": hbm, "unit": "GB/s", "frac": round(hbm_frac, 4),
                    "peak_source": hbm_src}
        roofline = {**head, "traffic": traffic(a, dom, n, dia, fixed),
                    "kernel": kernel_names[dom],
                    "ops_per_row": {"level": round(ops["level_avg"], 2), "update": ops["update"]},
                    "family_ms_per_solve": {k: round(v["ms"] / nprof, 3) for k, v in fam.items()},
                    "family_gops": gops, "family_frac": {k: round(g * 1e9 / peak, 4) for k, g in gops.items()},
                    "family_gbs": gbs, "family_hbm_frac": {k: round(g / hbm, 4) for k, g in gbs.items()},
                    "hbm_peak": hbm}
    else:
        achieved = d["bytes_per_launch"] / avg_s / 1e9
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(achieved / hbm, 4), "traffic": traffic(a, dom, n, dia, fixed),
                    "kernel": kernel_names[dom],
                    "peak_source": f"measured copy bandwidth ({hbm_src})",
                    "family_ms_per_solve": {k: round(v["ms"] / nprof, 3) for k, v in fam.items()},
                    "family_gbs": gbs}

    # plain PCG beside it, in the same arithmetic
    pcg = None
    if not a.no_pcg:
        psolver = sscg.Solver(A, method="pcg", tol=a.tol, maxit=20000, arith=a.arith)
        x.zero_()
        psolver.solve(b, x)
        pms, pres = timed(lambda: psolver.solve(b, x), max(1, min(a.steps, 3)))
        pprof = sscg.Solver(A, method="pcg", tol=a.tol, maxit=20000, arith=a.arith, profile=True)
        _, pres_p = timed(lambda: pprof.solve(b, x), 2)
        del pprof
        p0 = pres[-1]
        pcg_ms = max_over_ranks(pg, sum(pms)) / len(pms)
        pcg = dict(pcg_solve_ms=round(pcg_ms, 3), pcg_iters=p0.outer_iters, pcg_rel_res_true=p0.rel_res_true,
                   pcg_gbs=round(pcg_bytes(bm, p0.outer_iters) / (pcg_ms * 1e-3) / 1e9, 1),
                   pcg_yardstick_gbs=round(pcg_bytes(ym, p0.outer_iters) / (pcg_ms * 1e-3) / 1e9, 1),
                   speedup_vs_pcg=round(pcg_ms / ms_per_step, 4))
        if a.arith == "f64" and dia:
            pf = {}
            for key, cnt, fo in (("mpk", "n_mpk", ops["pcg_spmv"]), ("update", "n_update", ops["pcg_update"]),
                                 ("dir", "n_dir", ops["pcg_dir"])):
                t = sum(r.profile[f"t_{key}_ms"] for r in pres_p)
                c = sum(r.profile[cnt] for r in pres_p)
                if c:
                    pf[key] = round(fo * n / (t / c * 1e-3) / 1e9, 1)
            pcg["pcg_family_gops"] = pf
        # PFCG-NN (Algorithm 2), the paper's comparison solver, on the same kernels and arithmetic
        fsolver = sscg.Solver(A, method="pfcg", tol=a.tol, maxit=20000, arith=a.arith)
        x.zero_()
        fsolver.solve(b, x)
        fms, fres = timed(lambda: fsolver.solve(b, x), max(1, min(a.steps, 3)))
        pfcg_ms = max_over_ranks(pg, sum(fms)) / len(fms)
        pcg.update(pfcg_solve_ms=round(pfcg_ms, 3), pfcg_iters=fres[-1].outer_iters,
                   pfcg_rel_res_true=fres[-1].rel_res_true, speedup_vs_pfcg=round(pfcg_ms / ms_per_step, 4))
        del fsolver

    # the same FP64 solve with the block update's P and Q formed by FP64 FMAs
    fmau = None
    if fixed and not a.no_pcg:
        msolver = sscg.Solver(A, s=a.s, tol=a.tol, maxit=5000, arith=a.arith, fma_update=True)
        x.zero_()
        msolver.solve(b, x)
        mms, mres = timed(lambda: msolver.solve(b, x), 2)
        m_ms = max_over_ranks(pg, sum(mms)) / len(mms)
        mprof = sscg.Solver(A, s=a.s, tol=a.tol, maxit=5000, arith=a.arith, profile=True, fma_update=True)
        _, mres_p = timed(lambda: mprof.solve(b, x), 1)
        del mprof
        tu = sum(r.profile["t_update_ms"] for r in mres_p) / len(mres_p)
        fmau = {"fma_update_solve_ms": round(m_ms, 3), "fma_update_outer_iters": mres[-1].outer_iters,
                "fma_update_rel_res_true": mres[-1].rel_res_true,
                "fma_update_update_ms_per_solve": round(tu, 3),
                "fixed_update_speedup": round(m_ms / ms_per_step, 4)}
        if pcg:
            fmau["fma_update_speedup_vs_pcg"] = round(pcg["pcg_solve_ms"] / m_ms, 4)
        del msolver

    # the same solve and PCG in double-float (pairs of FP32, about 48 bits, FP32 exponent range)
    df = None
    if a.arith == "f64" and not a.no_df64:
        dsolver = sscg.Solver(A, s=a.s, tol=a.tol, maxit=5000, arith="df64")
        x.zero_()
        dsolver.solve(b, x)
        dms, dres = timed(lambda: dsolver.solve(b, x), 2)
        dp = sscg.Solver(A, method="pcg", tol=a.tol, maxit=20000, arith="df64")
        x.zero_()
        dp.solve(b, x)
        dpms, dpres = timed(lambda: dp.solve(b, x), 2)
        d_ms = max_over_ranks(pg, sum(dms)) / len(dms)
        dp_ms = max_over_ranks(pg, sum(dpms)) / len(dpms)
        df = {"df64_solve_ms": round(d_ms, 3), "df64_outer_iters": dres[-1].outer_iters,
              "df64_rel_res_true": dres[-1].rel_res_true, "df64_pcg_solve_ms": round(dp_ms, 3),
              "df64_speedup_vs_pcg": round(dp_ms / d_ms, 4),
              "df64_note": "double-float: pairs of FP32 (about 48 significant bits, FP32 exponent range) on the "
                           "FP32 units; narrower than FP64, reported for comparison only"}
        del dsolver, dp

    # the block sizes of the workload's definition, s in {1, 2, 4, 6, 8}: one
    # warm-up and two timed solves each (after the timed region)
    sweep = {}
    if not a.no_sweep:
        for sv in (1, 2, 4, 6, 8):
            if sv == a.s:
                sweep[str(sv)] = dict(ms=round(ms_per_step, 3), outer=r0.outer_iters, rel_res_true=r0.rel_res_true,
                                      status=r0.status, true_res_below_tol=bool(r0.rel_res_true <= a.tol))
                continue
            ssolver = sscg.Solver(A, s=sv, tol=a.tol, maxit=5000, arith=a.arith, fused_mpk=a.fused_mpk,
                                  fma_update=a.fma_update)
            x.zero_()
            ssolver.solve(b, x)
            sms, sres = timed(lambda: ssolver.solve(b, x), 2)
            sweep[str(sv)] = dict(ms=round(max_over_ranks(pg, sum(sms)) / len(sms), 3), outer=sres[-1].outer_iters,
                                  rel_res_true=sres[-1].rel_res_true, status=sres[-1].status,
                                  true_res_below_tol=bool(sres[-1].rel_res_true <= a.tol))
            del ssolver

    # end to end through the public API with host buffers
    bh = torch.from_numpy(sysm["b"]).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    hsolver = sscg.Solver(A, s=a.s, tol=a.tol, maxit=5000, arith=a.arith, host_vectors=True,
                          fused_mpk=a.fused_mpk, fma_update=a.fma_update)
    xh.zero_()
    hsolver.solve(bh, xh)
    e2e_t = []
    for _ in range(max(1, min(a.steps, 3))):
        xh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hr = hsolver.solve(bh, xh)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(pg, sum(e2e_t) / len(e2e_t))
    e2e = {"value": round(sum_over_ranks(pg, sstep_bytes(bm, hr.outer_iters)) / e2e_s / 1e9, 1), "unit": "GB/s",
           "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 8 * n, "ms_per_step": round(e2e_s * 1e3, 3)}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        o = oracle_sample(sysm, a.s, a.cpu_seconds, a.tol)
        per = (sstep_bytes(ym, o["steps"]) - ym["init"] - ym["final"]) / o["steps"]
        cpu = {"value": round(per * o["steps"] / o["seconds"] / 1e9, 3), "unit": "GB/s", "cores": o["threads"],
               "kind": "oracle",
               "sample": f"{o['steps']} outer steps of the same s={a.s} solve (tol 0), FP64 C oracle, "
                         f"{o['seconds']:.1f} s; bytes: the oracle's own (CSR with FP64 values, FP64 vectors, "
                         "A U and A P stored), outer steps only"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": a.arith, "data": "synthetic",
            "config": {"workload": workload_name(a.N, a.s, a.arith), "n": n, "nnz": nnz, "s": a.s,
                       "basis": "monomial", "preconditioner": "jacobi", "tol": a.tol,
                       "matrix_format": "diagonal form (7 offsets, presence mask)" if dia else "csr",
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 ({kernel_bytes_solve / max(r0.outer_iters, 1) / 1e9:.2f} GB "
                             "moved per outer step, working set > 4 GB); no flush needed"},
            "value_definition": "bytes the solve's kernels move (their algorithmic byte model, V = 8 n) per second "
                                "of device time; cannot exceed the copy bandwidth",
            "value_yardstick_gbs": round(value_yard, 1),
            "solve_ms": round(ms_per_step, 3), "solve_ms_steps": [round(t, 3) for t in ms],
            "outer_iters": r0.outer_iters, "equiv_iters": r0.equiv_iters,
            "status": r0.status, "rel_res_recursive": r0.rel_res_recursive, "rel_res_true": r0.rel_res_true,
            "yardstick_bytes_per_solve": yard_solve, "kernel_bytes_per_solve": kernel_bytes_solve,
            "wall_s_timed": round(t_wall, 3),
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(sum(r.profile["kernel_launches"] for r in res)),
            "clocks": clk, "cpu_baseline": cpu,
        }
        if pcg:
            line.update(pcg)
        if fmau:
            line.update(fmau)
        if df:
            line.update(df)
        if sweep:
            line["s_sweep"] = sweep
        print(json.dumps(line), flush=True)
    barrier(pg)


BATCH_METRIC = "batched s-step PCG serving: p50/p99 per-system latency and right-hand sides solved per second"


def batch_bytes(n, nnz, vbytes, R, s, outer):
    """Algorithmic bytes of one system's batched solve (df64 vectors, V = 8n):
    per level M + V (1/diag) + R V (u_j read, A u_j written) + R V more when
    j < s-1 (u_{j+1} written); per update R (6s + 6) V."""
    V = 8 * n
    M = 4 * (n + 1) + nnz * (4 + vbytes)
    levels = sum(M + V + R * V * (2 + (1 if j < s - 1 else 0)) for j in range(s))
    return outer * (levels + R * (6 * s + 6) * V)


def run_batch(a, world, rank, local, pg):
    """The serving mix: a.batch_systems seeded systems (7-/27-point stencils
    and variable-coefficient fields on 32^3..160^3 grids, 1..8 right-hand
    sides each) solved together by the batched kernels, timed over
    a.steps solves; the same solves one at a time through sscg_solve beside
    it.  Each rank solves its own mix (seeded by rank): replicas."""
    import multiprocessing as mp

    from paper_2501_03743_gb300 import inputs

    spec = inputs.batch_spec(a.batch_systems, seed=2025 + rank, nmin=a.batch_nmin, nmax=a.batch_nmax)
    var_idx = [k for k, e in enumerate(spec) if e["kind"] == "varcoef7"]
    t0 = time.perf_counter()
    var_csr = []
    if var_idx:  # the fields are built on the host cores, before any CUDA call
        with mp.get_context("spawn").Pool(max(1, min(len(var_idx), os.cpu_count() or 4))) as pool:
            var_csr = pool.map(inputs.batch_csr, [spec[k] for k in var_idx])
    import torch

    if rank == 0:
        from paper_2501_03743_gb300 import build

        build.build()
    barrier(pg)
    torch.cuda.set_device(local)
    from paper_2501_03743_gb300 import sscg

    ctx = sscg.Context()
    mats, sizes = [], []
    for k, e in enumerate(spec):
        if e["kind"] == "varcoef7":
            rp, c, v = var_csr[var_idx.index(k)]
        else:
            rp, c, v = inputs.stencil_torch(e["kind"], e["N"], "cuda")
        mats.append(sscg.Matrix(ctx, rp, c, v))
        sizes.append((mats[-1].n, mats[-1].nnz, 4 if mats[-1].props()["values_exact_fp32"] else 8))
        del rp, c, v
    var_csr = None
    t_gen = time.perf_counter() - t0
    R = [e["nrhs"] for e in spec]
    B = [ctx.uniform(R[k] * mats[k].n, 7000 + k).view(R[k], mats[k].n) for k in range(len(spec))]
    X = [torch.zeros_like(b) for b in B]
    t0 = time.perf_counter()
    plan = sscg.BatchSolver(mats, R, s=a.s, tol=a.tol, maxit=5000, arith=a.arith, tune=not a.no_tune,
                            persistent=a.persistent, fma_update=a.fma_update)
    t_plan = time.perf_counter() - t0
    props = plan.props()

    # the blocks of every right-hand side: 2 (2s + 1) columns, x and r, FP64
    ws = sum(n * R[k] * (2 * (2 * a.s + 1) + 2) * 8 for k, (n, _, _) in enumerate(sizes))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda") if ws <= L2_BYTES else None

    def one():
        for x in X:
            x.zero_()
        if flush is not None:
            flush.fill_(1.0)  # evict the previous solve's lines from L2
        torch.cuda.synchronize()
        return plan.solve(B, X)

    for _ in range(a.warmup):
        one()
    barrier(pg)
    clocks = Clocks(local)
    clocks.start()
    runs, launches = [], 0
    for _ in range(a.steps):
        runs.append(one())
        launches += plan.props()["launches"]  # kernels of that solve, graph nodes included
    clk = clocks.stop()
    barrier(pg)
    ms = [r.solve_ms for r in runs]
    lat = np.concatenate([r.latency_ms for r in runs])
    last = runs[-1]
    outer = [sy.outer_iters for sy in last.systems]
    total_rhs = sum(R)
    solve_ms = max_over_ranks(pg, statistics.median(ms))
    value = sum_over_ranks(pg, total_rhs) / (solve_ms * 1e-3)
    byts = sum(batch_bytes(n, nnz, vb, R[k], a.s, outer[k]) for k, (n, nnz, vb) in enumerate(sizes))

    seq = None
    if not a.no_seq:
        solvers = [sscg.Solver(m, s=a.s, tol=a.tol, maxit=5000, arith=a.arith) for m in mats]
        xs = [torch.zeros(m.n, dtype=torch.float64, device="cuda") for m in mats]
        # warm every solver once, then time all right-hand sides one by one
        for k in range(len(mats)):
            solvers[k].solve(B[k][0], xs[k])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        worst = 0
        for k in range(len(mats)):
            for r in range(R[k]):
                xs[k].zero_()
                res = solvers[k].solve(B[k][r], xs[k])
                worst = max(worst, res.status)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        seq_ms = e0.elapsed_time(e1)
        seq = {"seq_ms": round(seq_ms, 3), "seq_status": worst, "speedup_vs_sequential": round(seq_ms / solve_ms, 3)}
        del solvers, xs

    cpu = None
    if rank == 0:
        # the oracle beside it: the mix's smallest system, each of its right-hand sides
        # solved to the same tolerance by the FP64 CPU oracle's s-step PCG on the host
        # cores, scaled to the whole mix by the algorithmic bytes of the solves (the
        # byte model of this line: the sample's bytes at the oracle's own step counts,
        # the mix's at the device's)
        import oracle

        k0 = min(range(len(spec)), key=lambda k: sizes[k][0])
        Mo = oracle.as_matrix(dict(zip(("rowptr", "col", "val"), inputs.batch_csr(spec[k0]))))
        t0 = time.perf_counter()
        cpu_steps = 0
        for r in range(R[k0]):
            cpu_steps = max(cpu_steps, oracle.pcgs(Mo, B[k0][r].cpu().numpy(), a.s, tol=a.tol, maxit=5000).iters)
        t_cpu = time.perf_counter() - t0
        n0, nnz0, vb0 = sizes[k0]
        rate = batch_bytes(n0, nnz0, vb0, R[k0], a.s, cpu_steps) / t_cpu  # oracle bytes per second
        cpu = {"value": round(total_rhs / (byts / rate), 3), "unit": "rhs/s", "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": f"system {k0} of the mix ({spec[k0]['kind']} {spec[k0]['N']}^3, {R[k0]} right-hand "
                         f"sides, the smallest, {cpu_steps} outer steps): {t_cpu:.2f} s, "
                         f"{rate / 1e9:.2f} GB/s by the byte model; the whole mix's {byts / 1e9:.0f} GB at that "
                         f"rate: {byts / rate:.0f} s"}
        peak, src = hbm_peak()
        eff = byts / (statistics.median(ms) * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(eff, 1), "peak": peak, "unit": "GB/s", "frac": round(eff / peak, 4),
                "traffic": None, "kernel": "whole batched solve (k_bp_level, k_bp_solve, k_bp_update; "
                                           "algorithmic bytes of every system's levels and updates)",
                "peak_source": src}
    if rank == 0:
        classes = {}
        for k, (n, _, _) in enumerate(sizes):
            cls = 0 if n < 1 << 16 else (1 if n < 1 << 19 else (2 if n < 1 << 21 else 3))
            classes.setdefault(str(cls), props["tile_rows"][k])
        line = {
            "metric": BATCH_METRIC, "value": round(value, 2), "unit": "rhs/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(solve_ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": a.arith, "data": "synthetic",
            "config": {"workload": f"serving mix: {len(spec)} systems (7-/27-point stencils, variable-coefficient "
                                   f"fields sigma in {{0.5,1,2,3}}) on {a.batch_nmin}^3..{a.batch_nmax}^3 grids, "
                                   f"1..8 seeded RHS each "
                                   f"({total_rhs} RHS, {sum(n for n, _, _ in sizes):,} rows), s={a.s} monomial, "
                                   f"Jacobi, tol {a.tol}, x0=0",
                       "systems": len(spec), "rhs": total_rhs, "s": a.s, "tol": a.tol,
                       "parallelism": f"replicas x{world}",
                       "l2": (f"working set {ws / 1e9:.2f} GB (the mix's blocks), above L2; no flush needed"
                              if ws > L2_BYTES else
                              f"working set {ws / 1e9:.3f} GB fits L2: a {L2_FLUSH_BYTES >> 20} MiB buffer is "
                              "written before every solve")},
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                           "p99": round(float(np.percentile(lat, 99)), 3), "max": round(float(lat.max()), 3),
                           "samples": int(lat.size)},
            "solve_ms": {"median": round(statistics.median(ms), 3), "min": round(min(ms), 3),
                         "max": round(max(ms), 3)},
            "status": last.status, "max_rel_res_true": max(sy.rel_res_true for sy in last.systems),
            "max_outer_iters": max(outer),
            "effective_gbs": round(byts / (statistics.median(ms) * 1e-3) / 1e9, 1),
            "plan": {"grid": props["grid"], "cuda_graph": props["graph"], "tile_rows_by_class": classes,
                     "autotuned": not a.no_tune, "plan_s": round(t_plan, 2),
                     "mode": ("persistent cooperative launch" if a.persistent else
                              "per-phase launches over all systems, CUDA graph per outer step")},
            "gpu_launches": int(launches), "setup_s": round(t_gen, 1), "clocks": clk,
            "roofline": roof, "cpu_baseline": cpu,
        }
        if seq:
            line.update(seq)
        print(json.dumps(line), flush=True)
    barrier(pg)


MIXED_METRIC = "mixed-precision s-step PCG: 27-point 192^3 to rel. residual 1e-10, error vs the FP64 oracle"


def run_mixed27(a, world, rank, local, pg):
    """27-point stencil on 192^3 (a.N overrides), mixed precision (FP32 values
    and basis, FP64 Gram sums, P, AP, x, r, FP64 true-residual replacement
    every outer step) to 1e-10, beside the FP64 path to the same tolerance.
    The cpu_baseline leg solves the same system with the FP64 CPU oracle's PCG
    (timed on the host cores); its solution is also what the GPU solutions'
    error is measured against."""
    import torch

    from paper_2501_03743_gb300 import inputs
    import oracle

    N = a.N if a.N != 256 else 192
    sysm = inputs.system("poisson27", N, seed=rank)
    n, nnz = sysm["n"], len(sysm["col"])
    t0 = time.perf_counter()
    ref = oracle.pcg(oracle.as_matrix(sysm), sysm["b"], tol=1e-10, maxit=20000)  # host cores, before CUDA
    t_oracle = time.perf_counter() - t0
    if rank == 0:
        from paper_2501_03743_gb300 import build

        build.build()
    barrier(pg)
    torch.cuda.set_device(local)
    from paper_2501_03743_gb300 import sscg

    ctx = sscg.Context()
    A = sscg.Matrix(ctx, sysm["rowptr"], sysm["col"], sysm["val"])
    b = torch.from_numpy(sysm["b"]).cuda()
    x = torch.zeros_like(b)
    out = {}
    for name, kw in (("mixed", dict(arith="mixed", replace_every=1)), ("f64", dict(arith="f64"))):
        solver = sscg.Solver(A, s=a.s, tol=1e-10, maxit=5000, profile=True, **kw)
        for _ in range(max(1, a.warmup)):
            x.zero_()
            solver.solve(b, x)
        ms, res, nl = [], None, 0
        for _ in range(max(1, a.steps)):
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            res = solver.solve(b, x)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            nl += res.profile["kernel_launches"]
        xs = x.cpu().numpy()
        if name == "mixed":
            sv = a.s
            # bytes per timed record (the mixed driver times the s levels, the Gram pass and
            # the update + residual replacement of an outer step as one record each)
            # FP64 operations per timed record (the s levels, the Gram pass, the update with the
            # replacement; residual replaced every step, so no A P): levels 3 a row each (A U
            # widened to FP64); Gram s(s+1)/2 + s + s^2 + s FMAs and s widenings; update s^2 + s
            # FMAs and s widenings; replacement (neighbour sum on the integer units) an FMA, r0 - y,
            # ||r||^2 and B^-1 r rounded to FP32: 5
            fam_ops = {"mpk": 3 * sv * n, "dir": (sv * (sv + 1) // 2 + 3 * sv + sv * sv) * n,
                       "update": (sv * sv + 2 * sv + 5) * n}
            names = {"mpk": "k_mx_level x s (diagonal-form SpMV of the FP32 basis, AU widened to FP64)",
                     "dir": "k_gram (G, C = P_old^T (A U), m and q of the direct-Gram blocks, FP64 sums)",
                     "update": "k_mx_update + k_mx_replace (P, x; r = r0 - A(x - x0) in FP64)"}
            mixed_roof = family_alu_roofline(res, fam_ops, names, torch.cuda.get_device_properties(local)
                                             .multi_processor_count)
        out[name] = dict(ms=statistics.median(ms), outer=res.outer_iters, status=res.status, launches=nl,
                         rel_res_true=res.rel_res_true,
                         err_vs_oracle=float(np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x)),
                         err_vs_x_true=float(np.linalg.norm(xs - sysm["x_true"]) / np.linalg.norm(sysm["x_true"])))
    m = out["mixed"]
    if rank == 0:
        line = {"metric": MIXED_METRIC, "value": round(m["ms"], 3), "unit": "ms", "n_gpus": world,
                "steps": a.steps, "warmup": max(1, a.warmup), "ms_per_step": round(m["ms"], 3), "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "mixed (fp32 basis and values, fp64 accumulation)",
                "data": "synthetic",
                "config": {"workload": f"poisson27 {N}^3 (n={n:,}, nnz={nnz:,}), Jacobi, s={a.s} monomial, "
                                       "b=A x_true, x0=0, tol 1e-10, true-residual replacement every outer step",
                           "parallelism": f"replicas x{world}"},
                "mixed": {k: (round(v, 3) if k == "ms" else v) for k, v in m.items()},
                "f64": {k: (round(v, 3) if k == "ms" else v) for k, v in out["f64"].items()},
                "speedup_mixed_vs_f64": round(out["f64"]["ms"] / m["ms"], 3),
                "roofline": mixed_roof,
                "gpu_launches": int(m["launches"]),
                "cpu_baseline": {"value": round(t_oracle * 1e3, 1), "unit": "ms", "cores": oracle.num_threads(),
                                 "kind": "oracle",
                                 "sample": f"the whole solve: FP64 CPU oracle PCG to 1e-10, {ref.iters} iterations"}}
        print(json.dumps(line), flush=True)
    barrier(pg)


CHEB_METRIC = "Chebyshev-basis s-step PCG with network vs Lanczos intervals: time to 1e-8 incl. the interval"


def run_cheb(a, world, rank, local, pg):
    """Variable-coefficient 7-point 128^3 fields with sigma in {0.5, 1, 2, 3}:
    the Chebyshev-basis solve at s = 8 and 12 with its interval from the
    trained spectral-bound network vs from 20 Lanczos steps (the library's
    fallback), time including the interval; monomial s = 8 / 12 beside it.
    The network is trained on the device first (seeded recipe)."""
    import torch

    from paper_2501_03743_gb300 import inputs

    N = a.N if a.N != 256 else 128
    if rank == 0:
        from paper_2501_03743_gb300 import build

        build.build()
    barrier(pg)
    torch.cuda.set_device(local)
    from paper_2501_03743_gb300 import spectral, sscg

    ctx = sscg.Context()
    t0 = time.perf_counter()
    samples = spectral.default_samples(seeds_per=6)
    samples += [spectral.Sample("varcoef7", M, 3.0, ell, 700 + q)
                for q, (M, ell) in enumerate([(32, 4.0), (48, 2.0), (64, 8.0), (96, 4.0), (128, 4.0), (80, 2.0)])]
    X, T = spectral.dataset(ctx, samples)
    net, hist = spectral.fit(ctx, X, T, hidden=64, epochs=4000, lr=3e-3, seed=0)
    blob = net.blob()
    t_train = time.perf_counter() - t0
    rows = []
    for q, sig in enumerate((0.5, 1.0, 2.0, 3.0)):
        c = inputs.varcoef7(N, sig, 5000 + q)
        A = sscg.Matrix(ctx, *c)
        bt = torch.from_numpy(inputs.matvec(*c, inputs.uniform(91 + q, A.n))).cuda()
        x = torch.zeros_like(bt)

        def timed(fn):
            # a.warmup untimed calls, then the median of a.steps timed ones
            for _ in range(max(1, a.warmup)):
                fn()
            torch.cuda.synchronize()
            ts, out = [], None
            for _ in range(max(1, a.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                out = fn()
                e1.record(ctx.stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return out, statistics.median(ts)

        for s in (8, 12):
            row = {"sigma": sig, "s": s}
            for name in ("network", "lanczos", "monomial"):
                if name == "network":
                    A.set_bounds_model(net.h, blob)
                else:
                    A.set_bounds_model(net.h, None)
                basis = "monomial" if name == "monomial" else "chebyshev"
                solver = sscg.Solver(A, s=s, basis=basis, tol=1e-8, maxit=4000, profile=True)

                def go():
                    x.zero_()
                    return solver.solve(bt, x)

                r, ms = timed(go)
                row[name] = {"ms": round(ms, 3), "status": r.status, "outer": r.outer_iters,
                             "rel_res_true": r.rel_res_true, "launches": r.profile["kernel_launches"]}
                if name == "network" and sig == 3.0 and s == 8:
                    nn = A.n
                    # FP64 operations per timed record: s levels of a 7-point CSR row (7 FMAs, the
                    # Jacobi scale, the Chebyshev recurrence's 3); the Gram pass's s(s+1)/2 + s + s^2
                    # FMAs; the update's 2 s^2 + 2 s FMAs for P, AP, x, r and 3 for z and the norms
                    cheb_roof = family_alu_roofline(
                        r, {"mpk": 11 * s * nn, "dir": (s * (s + 1) // 2 + s + s * s) * nn,
                            "update": (2 * s * s + 2 * s + 3) * nn},
                        {"mpk": "k_level_gen x s (CSR SpMV, AU stored, Chebyshev recurrence)",
                         "dir": "k_gram (G, C, m of the direct-Gram blocks)",
                         "update": "k_update_ap (P, AP, x, r, z; s <= 8)"},
                        torch.cuda.get_device_properties(local).multi_processor_count)
                    cheb_roof["workload"] = f"sigma=3 field {N}^3, Chebyshev basis s=8, network interval"
                    cheb_csr = c
            A.set_bounds_model(net.h, None)
            (lo, hi), t_net = timed(lambda: net.bounds(A, blob))
            (llo, lhi), t_lz = timed(lambda: A.estimate_bounds(20))
            row["interval_ms"] = {"network": round(t_net, 3), "lanczos20": round(t_lz, 3)}
            row["interval"] = {"network": [lo, hi], "lanczos20": [llo, lhi]}
            rows.append(row)
        A.close()
    if rank == 0:
        # the oracle beside it: the two interval computations on the host cores for the
        # sigma = 3 field (features + forward pass of the same network, 20 Lanczos steps)
        import oracle

        Mo = oracle.as_matrix(dict(rowptr=cheb_csr[0], col=cheb_csr[1], val=cheb_csr[2]))
        st = net.state()
        t0 = time.perf_counter()
        f = oracle.features(Mo)
        oracle.mlp_forward(st["d"], st["h"], st["o"], st["theta"], ((f - st["x_mean"]) / st["x_std"])[None, :])
        t_net_cpu = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.lanczos_bounds(Mo, inputs.uniform(91, N ** 3), 20)
        t_lz_cpu = time.perf_counter() - t0
        ok = [r for r in rows if r["network"]["status"] == 0 and r["lanczos"]["status"] == 0]
        gain = [r["lanczos"]["ms"] / r["network"]["ms"] for r in ok]
        line = {"metric": CHEB_METRIC, "value": round(statistics.median(gain), 3) if gain else None,
                "unit": "x (Lanczos-interval time / network-interval time, median)", "n_gpus": world,
                "steps": max(1, a.steps), "warmup": max(1, a.warmup), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"varcoef7 {N}^3, k = exp(sigma g), sigma in {{0.5,1,2,3}}, Jacobi, "
                                       "Chebyshev basis s in {8,12}, tol 1e-8",
                           "training": f"{len(samples)} seeded systems at 8^3..128^3, labels from device "
                                       f"Lanczos, {len(hist)} Adam epochs, {t_train:.1f} s",
                           "parallelism": f"replicas x{world}"},
                "gpu_launches": int(sum(r["network"]["launches"] + r["lanczos"]["launches"] for r in rows)),
                "roofline": cheb_roof,
                "cpu_baseline": {"value": round(t_lz_cpu / t_net_cpu, 3),
                                 "unit": "x (oracle 20-step Lanczos time / oracle features + network time)",
                                 "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": f"sigma=3 field {N}^3: oracle features + forward {t_net_cpu * 1e3:.1f} ms, "
                                           f"oracle 20-step Lanczos {t_lz_cpu * 1e3:.1f} ms"},
                "rows": rows}
        print(json.dumps(line), flush=True)
    barrier(pg)


PEAKS_METRIC = "arithmetic throughput probes: operations per second over the device"


def probe_calibrated(ctx, kind, target_ms=100.0, iters_b=0):
    """Run a probe once short, then with the iteration count that takes about
    target_ms; best of three at that count."""
    ops, ms = ctx.probe_rate(kind, 256, iters_b if iters_b else 0)
    it = max(256, int(256 * target_ms / max(ms, 1e-3)))
    best = None
    for _ in range(3):
        r = ctx.probe_rate(kind, it, iters_b)
        best = r if best is None or r[0] > best[0] else best
    return best[0], best[1], it


def fp64_alu_peak(sm_count, sm_mhz):
    """FP64 operations per second at sm_mhz: the nominal 1.25 TFLOP/s of a
    GB300 at its 2070 MHz maximum SM clock is 2 FP64 FMAs per clock per SM
    (1.25e12 / 2 / 152 / 2.07e9 = 1.99)."""
    return 2.0 * sm_count * sm_mhz * 1e6


def run_peaks(a, world, rank, local, pg):
    """Each probe of include/sscg_probe.h for about 100 ms over a full-device
    grid (best of three), with the SM clock sampled meanwhile; the mixed probe
    runs DFMA and DMMA warps together with equal solo times to show whether
    the FP64 tensor instruction adds throughput to the FP64 FMA pipe."""
    import torch

    if rank == 0:
        from paper_2501_03743_gb300 import build

        build.build()
    barrier(pg)
    torch.cuda.set_device(local)
    from paper_2501_03743_gb300 import sscg

    ctx = sscg.Context()
    sm = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = Clocks(local)
    clocks.start()
    rates = {}
    for kind in ("dfma", "dadd", "dmul", "dmma", "ffma", "ialu", "imad", "imad_wide", "i2f64", "f2i64"):
        ops, ms, it = probe_calibrated(ctx, kind)
        rates[kind] = {"ops_per_s": ops, "ms": round(ms, 3), "iters": it}
    # equal solo times: the DMMA warps' iteration count scaled from the solo rates
    itf = rates["dfma"]["iters"]
    t_f = rates["dfma"]["ms"]
    itm = max(1, int(rates["dmma"]["iters"] * t_f / rates["dmma"]["ms"]))
    best = None
    for _ in range(3):
        r = ctx.probe_rate("dfma_dmma", itf, itm)
        best = r if best is None or r[0] > best[0] else best
    rates["dfma_dmma"] = {"ops_per_s": best[0], "ms": round(best[1], 3), "iters": [itf, itm],
                          "time_vs_solo": round(best[1] / t_f, 3)}
    clk = clocks.stop()
    # latency of the on-chip s x s solves (one warp, SM cycles), s = 2, 4, 8
    small = {str(s): {k: round(v, 1) for k, v in ctx.probe_small_solve(s, 200).items()} for s in (2, 4, 8)}
    if rank == 0:
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        per = {k: round(v["ops_per_s"] / (sm * mhz * 1e6), 3) for k, v in rates.items()}
        line = {"metric": PEAKS_METRIC, "value": round(rates["dfma"]["ops_per_s"] / 1e9, 1),
                "unit": "G FP64 FMA/s", "n_gpus": world, "steps": 3, "warmup": 1, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"full-device grid ({sm} SMs), independent dependency chains per thread, "
                                       "about 100 ms per probe, best of 3"},
                "rates_gops": {k: round(v["ops_per_s"] / 1e9, 2) for k, v in rates.items()},
                "per_sm_per_clock": per, "sm_count": sm, "detail": rates,
                "fp64_nominal_derived_gops_at_max_clock": round(fp64_alu_peak(sm, 2070.0) / 1e9, 1),
                "small_solve_cycles": small,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    barrier(pg)


def reference_arm(a, world, rank, pg):
    """The oracle timed as the reference arm: each step one bounded sample
    (a few outer steps) of the same solve on the host cores."""
    if rank != 0:
        return
    from paper_2501_03743_gb300 import inputs
    import oracle

    sysm = inputs.system("poisson7", a.N, seed=0)
    n, nnz = sysm["n"], len(sysm["col"])
    bm = yardstick(n, nnz, a.s)
    M = oracle.as_matrix(sysm)
    t0 = time.perf_counter()
    oracle.pcgs(M, sysm["b"], a.s, tol=0.0, maxit=1)
    one = time.perf_counter() - t0
    per_step_outer = max(1, min(50, int(8.0 / max(one, 1e-6))))
    for _ in range(a.warmup):
        oracle.pcgs(M, sysm["b"], a.s, tol=0.0, maxit=1)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.pcgs(M, sysm["b"], a.s, tol=0.0, maxit=per_step_outer)
        times.append(time.perf_counter() - t0)
    byts = sstep_bytes(bm, per_step_outer)
    value = byts * a.steps / sum(times) / 1e9
    line = {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(1e3 * sum(times) / a.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(a.N, a.s, "f64"), "n": n, "nnz": nnz, "s": a.s,
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"each step: {per_step_outer} outer steps of the s={a.s} solve, FP64 C oracle"},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
