#!/usr/bin/env python
"""Benchmark of the block ILU(k)-preconditioned BiCGSTAB hot path on one GB300.

One step = everything that depends on the matrix values, on the resident
inputs: backfill A -> A', block ILU factorization (Algorithm 4) with the
diagonal factorization U = D U' (Eq. 5), then BiCGSTAB from x0 = 0 toward a
true relative residual of 1e-8 with an iteration budget of --maxit (each
iteration: two preconditioner applies (Eq. 6, Algorithm 7) and two block
SpMVs).  The 128 x 128 x 64 workload (sigma = 2, accumulation 1e-3) does not
reach 1e-8 with ILU(1)-BiCGSTAB (neither does the CPU oracle), so on it a
step is the factorization plus exactly --maxit iterations; the line says
whether the solve converged.  The 16 x 16 x 8 workload, which converges, is
also timed to 1e-8 (``ms_to_tol_small``).  The symbolic phase (Algorithm 3)
depends on the pattern only; it runs once at set-up and its host time is
reported next to the step (``symbolic_ms``).

Output: one JSON line (rank 0).  ``value`` is milliseconds per step (lower is
better).  ``roofline`` reports the dominant kernel's algorithmic bytes per
launch divided by its mean CUDA-event duration over the timed region, against
the measured HBM copy bandwidth.  ``e2e`` repeats the step through the public
API from pinned host buffers (A's values and the right-hand side copied in,
x copied out, inside the timed region).  ``cpu_baseline`` is the CPU oracle
timed on a bounded sample of the same workload.

``--impl reference`` times the CPU oracle as the reference arm (no GPU use).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Block-ILU(k) BiCGSTAB ms to 1e-8 resid; trisolve/SpMV GB/s; FP32-prec vs FP64"
WORKLOAD = "grid128x128x64_7pt_b3"
FP64_PEAK_TFLOPS = 1.196  # measured FP64 FMA rate of this GB300 (FMA = 2 flops)
# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of the
# kernel as it stands (the summary under profiles/ gives the command); keyed by
# (workload, k, kernel).  The capture
# runs on the 96 x 96 x 48 case (the recipe's size rule); a solve streams each
# factor block once, so its traffic is scaled to the 128 x 128 x 64 launch by
# the algorithmic bytes.  Missing entries (no capture of the kernel as it
# stands) report null.
NCU_TRAFFIC = {
    ("grid128x128x64_7pt_b3", 1, "upper_solve"): 552320350,   # 1.052 x algorithmic
    ("grid128x128x64_7pt_b3", 1, "lower_solve"): 551958807,   # 1.051 x
    ("grid128x128x64_7pt_b3", 1, "diag_scale"): 100673612,    # 0.800 x (z stays in L2)
    ("grid128x128x64_7pt_b3", 1, "spmv"): 601747660,          # 0.991 x
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--b", type=int, default=0, help="block size for workloads without one (default 3)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=100)
    ap.add_argument("--chunk", type=int, default=0, help="trisolve rows per warp (0 = library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP32-preconditioner comparison")
    ap.add_argument("--no-c2", action="store_true", help="skip the brief b x k sweep of the 96 x 96 x 48 grid")
    ap.add_argument("--sweep", choices=["c2", "c3"], default=None,
                    help="instead of the bench line: one JSON line per configuration of the 96 x 96 x 48 "
                         "b x k sweep (c2) or of the 160 x 160 x 80 27-point ILU(2) case (c3)")
    ap.add_argument("--oracle", action="store_true",
                    help="with --sweep c2: add the CPU oracle's kernel times (one call each, one thread)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the step only (no small-case, FP32-kernel or precision sections)")
    ap.add_argument("--kernel-case", choices=["apply", "apply_f32", "spmv", "spmv_f32", "spmv_f32x"], default=None,
                    help="instead of the bench line: run one preconditioner apply or SpMV --reps times on "
                         "--workload (the small single-kernel case for profilers)")
    ap.add_argument("--reps", type=int, default=3)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def system(args):
    from paper_1703_01325_gb300.reservoir import WORKLOADS, reservoir_system
    cfg = dict(WORKLOADS[args.workload])
    if "b" not in cfg or args.b:
        cfg["b"] = args.b or cfg.get("b", 3)
    return reservoir_system(**cfg), cfg


def algorithmic_bytes(n, b, nnz_a, nnz_l, nnz_u, v=8):
    """Bytes a kernel must move at least once (values, indices, vectors)."""
    bb = b * b
    spmv = nnz_a * (v * bb + 4) + 4 * (n + 1) + 2 * n * b * 8            # A, x in, y out (FP64 vectors)
    lower = nnz_l * (v * bb + 4) + 4 * (n + 1) + 2 * n * b * 8            # L, r in, y out (FP64 vectors)
    diag = n * v * bb + 2 * n * b * 8                                     # D^-1, y in, z out
    upper = nnz_u * (v * bb + 4) + 4 * (n + 1) + 2 * n * b * 8            # U', z in, x out
    return dict(spmv=spmv, lower_solve=lower, diag_scale=diag, upper_solve=upper,
                apply=lower + diag + upper)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import statistics
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(S, k, gpu_iters, sample_iters=4):
    """The CPU oracle (single thread) on a bounded sample: the full symbolic
    phase and factorization plus `sample_iters` BiCGSTAB iterations, scaled to
    the iteration count of the measured solve."""
    import oracle
    t0 = time.perf_counter()
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, k)
    t1 = time.perf_counter()
    A1 = oracle.backfill(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci)
    F, D = oracle.factor(S.n, S.b, prp, pci, A1)
    t2 = time.perf_counter()
    oracle.bicgstab(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci, F, D, S.rhs, tol=1e-300,
                    maxit=sample_iters)
    t3 = time.perf_counter()
    # bicgstab also pays one SpMV for r0 and one for the true residual
    per_it = (t3 - t2) / sample_iters
    factor_ms = (t2 - t1) * 1e3
    value = factor_ms + per_it * 1e3 * max(gpu_iters, 1)
    t4 = time.perf_counter()
    oracle.spmv(S.n, S.b, S.row_ptr, S.col_idx, S.vals, S.rhs)
    t5 = time.perf_counter()
    oracle.apply(S.n, S.b, prp, pci, F, D, S.rhs)
    t6 = time.perf_counter()
    return {"value": round(value, 1), "unit": "ms", "cores": 1, "kind": "oracle", "estimate": True,
            "sample_iters": sample_iters, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "kernels_ms": {"symbolic": round(1e3 * (t1 - t0), 1), "factor": round(factor_ms, 1),
                           "spmv": round(1e3 * (t5 - t4), 1), "apply": round(1e3 * (t6 - t5), 1)},
            "sample": (f"oracle factorization of the full matrix ({factor_ms:.0f} ms) + {sample_iters} "
                       f"BiCGSTAB iterations ({per_it * 1e3:.0f} ms each), scaled to {gpu_iters} iterations; "
                       f"symbolic {1e3 * (t1 - t0):.0f} ms not counted")}


def oracle_kernel_times(S, k):
    """One call of each CPU oracle kernel (single thread) on the full system:
    symbolic phase, backfill + factorization, SpMV, apply."""
    import oracle
    t0 = time.perf_counter()
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, k)
    t1 = time.perf_counter()
    A1 = oracle.backfill(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci)
    F, D = oracle.factor(S.n, S.b, prp, pci, A1)
    t2 = time.perf_counter()
    oracle.spmv(S.n, S.b, S.row_ptr, S.col_idx, S.vals, S.rhs)
    t3 = time.perf_counter()
    oracle.apply(S.n, S.b, prp, pci, F, D, S.rhs)
    t4 = time.perf_counter()
    return {"kind": "oracle", "cores": 1, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "kernels_ms": {"symbolic": round(1e3 * (t1 - t0), 1), "factor": round(1e3 * (t2 - t1), 1),
                           "spmv": round(1e3 * (t3 - t2), 1), "apply": round(1e3 * (t4 - t3), 1)},
            "sample": "one call of each oracle kernel on the full system"}


def cpu_model() -> str:
    """The host CPU's model name (as /proc/cpuinfo or lscpu give it)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def replica_group(backend: str, device=None):
    """(dist, world, rank, local) from the launcher's environment.  With more
    than one rank every rank solves its own copy of the workload (replicas:
    the ILU(k) recurrences do not shard), so the group only times them."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world <= 1:
        return None, 1, 0, local
    import torch.distributed as dist
    kw = {"device_id": device} if device is not None else {}
    dist.init_process_group(backend, **kw)
    return dist, world, rank, local


def max_over_ranks(value: float, dist, device="cpu") -> float:
    """The largest value over all ranks (the slowest replica's step time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    S, cfg = system(args)
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, args.k)
    iters_ref = args.maxit  # the workload does not converge within the budget
    sample_iters = 2

    def step():
        t1 = time.perf_counter()
        A1 = oracle.backfill(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci)
        F, D = oracle.factor(S.n, S.b, prp, pci, A1)
        t2 = time.perf_counter()
        oracle.bicgstab(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci, F, D, S.rhs, tol=1e-300,
                        maxit=sample_iters)
        t3 = time.perf_counter()
        return (t2 - t1) * 1e3 + (t3 - t2) / sample_iters * 1e3 * iters_ref

    for _ in range(args.warmup):
        step()
    vals = [step() for _ in range(args.steps)]
    ms = sum(vals) / len(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": round(ms, 1), "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "k": args.k, "tol": args.tol, "maxit": args.maxit, **cfg,
                   "step": "backfill + factor + BiCGSTAB iterations up to maxit"},
        "estimate": True,
        "cpu_baseline": {"value": round(ms, 1), "unit": "ms", "cores": 1, "kind": "oracle", "estimate": True,
                         "sample_iters": sample_iters, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                         "sample": f"per step: full factorization + {sample_iters} BiCGSTAB iterations timed, "
                                   f"the iterations scaled to {iters_ref}: the value is an estimate"},
        "e2e": {"value": round(ms, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def oracle_solution(S, k, tol=1e-12, maxit=600):
    """The CPU oracle's FP64 solution of S (symbolic, backfill, factor and
    BiCGSTAB toward `tol`, one thread): the reference every GPU solution's
    error is stated against."""
    import oracle
    t0 = time.perf_counter()
    prp, pci, _ = oracle.symbolic(S.n, S.row_ptr, S.col_idx, k)
    F, D = oracle.factor(S.n, S.b, prp, pci, oracle.backfill(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci))
    x, it, rr, st = oracle.bicgstab(S.n, S.b, S.row_ptr, S.col_idx, S.vals, prp, pci, F, D, S.rhs, tol=tol,
                                    maxit=maxit)
    return {"x": x, "iters": int(it), "true_relres": float(rr), "status": int(st),
            "seconds": round(time.perf_counter() - t0, 1)}


def rel_err(x, ref) -> float:
    """||x - ref|| / ||ref|| (2-norms, x a device or host vector)."""
    import numpy as np
    xv = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    return float(np.linalg.norm(xv - ref) / np.linalg.norm(ref))


def fp64_issue_ceiling(P, b, sms, sm_mhz, cycles_per_instr=19.0):
    """Lower bound on each FP64 sweep's time from FP64 issue alone: the solve
    kernel spreads a row's blocks over G groups of b lanes (the fewest that
    hold the widest row, at least a quarter of the 32 // b), each lane does b
    DFMAs per block it takes and log2(G) shuffle-add steps sum the groups,
    so a row of m blocks costs ceil(m / G) * b + log2(G) FP64 warp
    instructions; this part issues one FP64 warp instruction per ~19 cycles
    per SM (measured), with the rows spread evenly over the SMs."""
    import math
    import numpy as np
    e = P.export()
    rp, ci = e["row_ptr"], e["col_idx"]
    rows = np.repeat(np.arange(P.n), np.diff(rp))
    gfull = 32 if b == 1 else 16 if b == 2 else 8 if b <= 4 else 4
    out = {}
    for name, mask in (("lower_solve", ci < rows), ("upper_solve", ci > rows)):
        m = np.bincount(rows[mask], minlength=P.n)
        need = int(m.max()) if P.n else 0
        g = gfull // 4 if need <= gfull // 4 else gfull // 2 if need <= gfull // 2 else gfull
        instr = np.ceil(m / g) * b + math.log2(g)
        per_sm = instr.sum() / sms
        out[name] = {"groups": g, "fp64_instr_per_row": round(float(instr.mean()), 3),
                     "ceiling_us": round(per_sm * cycles_per_instr / sm_mhz, 1)}
    return out


def ms_to_tol_c2(B, dev, stream, b=3, k=1, reps=3, tol=1e-8, ref=None):
    """Factor + FP64 BiCGSTAB from x0 = 0 to a true relative residual of 1e-8
    on the 96 x 96 x 48 7-point workload (b = 3, ILU(1); inputs larger than
    L2), timed like the step (CUDA events, median of `reps`), with the
    solution's error against the CPU oracle's FP64 solution."""
    import torch
    from paper_1703_01325_gb300.reservoir import WORKLOADS, reservoir_system
    S = reservoir_system(b=b, **WORKLOADS["grid96x96x48_7pt"])
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
    rp, ci = torch.from_numpy(S.row_ptr).to(dev), torch.from_numpy(S.col_idx).to(dev)
    vals, rhs = torch.from_numpy(S.vals.reshape(-1)).to(dev), torch.from_numpy(S.rhs).to(dev)
    F = B.new_factors(P, b, dev)
    fw = B.workspace(P.factor_workspace_bytes(b), dev)
    sw = B.workspace(P.bicgstab_workspace_bytes(b), dev)
    x = torch.zeros_like(rhs)
    runs = []
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, finfo = B.bilu_factor(P, b, vals, F, fw)
        x.zero_()
        _, info = B.bicgstab_solve(P, (S.n, b, rp, ci, vals), F, rhs, x=x, tol=tol, maxit=2000, work=sw)
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            runs.append((e0.elapsed_time(e1), finfo.ms, info))
    runs.sort(key=lambda t: t[0])
    ms, fms, info = runs[len(runs) // 2]
    out = {"workload": "grid96x96x48_7pt", "b": b, "k": k, "tol": tol, "ms": round(ms, 2),
           "factor_ms": round(fms, 2), "iters": info.iters, "true_relres": info.true_relres,
           "status": info.status, "l2": "inputs larger than L2 (A values %.0f MB)" % (S.nnzb * b * b * 8 / 1e6)}
    if ref is None:
        ref = oracle_solution(S, k)
    out["x_rel_err_vs_oracle"] = rel_err(x, ref["x"])
    out["oracle_reference"] = {k2: ref[k2] for k2 in ("iters", "true_relres", "status", "seconds")}
    P.close()
    return out


def ms_to_tol_small(B, dev, stream, reps=5):
    """Factor + BiCGSTAB to 1e-8 on the 16 x 16 x 8, b = 3, ILU(1) workload,
    which converges (launch/latency bound: it fits in L2)."""
    import torch
    from paper_1703_01325_gb300.reservoir import WORKLOADS, reservoir_system
    S = reservoir_system(**WORKLOADS["grid16x16x8_7pt_b3"])
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, 1).upload()
    rp, ci = torch.from_numpy(S.row_ptr).to(dev), torch.from_numpy(S.col_idx).to(dev)
    vals, rhs = torch.from_numpy(S.vals.reshape(-1)).to(dev), torch.from_numpy(S.rhs).to(dev)
    F = B.new_factors(P, S.b, dev)
    fw = B.workspace(P.factor_workspace_bytes(S.b), dev)
    sw = B.workspace(P.bicgstab_workspace_bytes(S.b), dev)
    x = torch.zeros_like(rhs)
    times, info = [], None
    for r in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.bilu_factor(P, S.b, vals, F, fw)
        x.zero_()
        _, info = B.bicgstab_solve(P, (S.n, S.b, rp, ci, vals), F, rhs, x=x, tol=1e-8, maxit=1000, work=sw)
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    times.sort()
    return {"workload": "grid16x16x8_7pt_b3", "k": 1, "ms": round(times[len(times) // 2], 3),
            "iters": info.iters, "true_relres": info.true_relres, "status": info.status}


def precision_compare(B, dev, stream, cases=((2, 1), (4, 1)), tol=1e-8, with_oracle=True):
    """Two FP32-preconditioner solvers against the plain FP64 solve
    (bilu_factor + bicgstab_solve), all from x0 = 0 to a true relative
    residual of `tol`, on the 96 x 96 x 48 7-point workload at block sizes b
    and fill levels k: "mixed" = FP32-stored preconditioner and FP32 SpMV
    inside FP64 iterative refinement (bilu_factor_f32 + bicgstab_solve_mixed);
    "f32prec" = FP64 BiCGSTAB with the FP32-stored preconditioner
    (bilu_factor_f32 + bicgstab_solve_f32prec); "f32prec_from_fp64" = the same
    with the FP64 factors rounded to FP32 (bilu_factor + bilu_convert_f32);
    "fp64_gmres20" = the FP64 preconditioner in restarted GMRES(20), the
    solver of the paper's experiments (bilu_factor + gmres_solve).
    Times include the factorization.  Each solution's error is stated against
    the CPU oracle's FP64 solution of the same system (BiCGSTAB to 1e-12)."""
    import torch
    from paper_1703_01325_gb300.reservoir import WORKLOADS, reservoir_system
    out = []
    for b, k in cases:
        S = reservoir_system(b=b, **WORKLOADS["grid96x96x48_7pt"])
        P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k).upload()
        rp, ci = torch.from_numpy(S.row_ptr).to(dev), torch.from_numpy(S.col_idx).to(dev)
        vals, rhs = torch.from_numpy(S.vals.reshape(-1)).to(dev), torch.from_numpy(S.rhs).to(dev)
        A = (S.n, b, rp, ci, vals)
        F = B.new_factors(P, b, dev)
        F32 = torch.empty(max(P.factor_bytes_f32(b) // 4, 1), dtype=torch.float32, device=dev)
        fw = B.workspace(P.factor_workspace_bytes(b), dev)
        sw = B.workspace(P.bicgstab_workspace_bytes(b), dev)
        mw = B.workspace(P.bicgstab_mixed_workspace_bytes(b), dev)
        vals32 = B.bilu_convert_f32(vals)
        x64, x32 = torch.zeros_like(rhs), torch.zeros_like(rhs)

        def fp64():
            B.bilu_factor(P, b, vals, F, fw)
            x64.zero_()
            return B.bicgstab_solve(P, A, F, rhs, x=x64, tol=tol, maxit=5000, work=sw)[1]

        def mixed():
            B.bilu_convert_f32(vals, vals32)
            B.bilu_factor_f32(P, b, vals, F32, fw)
            x32.zero_()
            return B.bicgstab_solve_mixed(P, A, vals32, F32, rhs, x=x32, tol=tol, maxit=5000, inner_tol=1e-3,
                                          inner_maxit=300, work=mw)[1]

        def f32prec():
            B.bilu_factor_f32(P, b, vals, F32, fw)
            xp.zero_()
            return B.bicgstab_solve_f32prec(P, A, F32, rhs, x=xp, tol=tol, maxit=5000, work=sw)[1]

        def f32prec_from_fp64():
            B.bilu_factor(P, b, vals, F, fw)
            B.bilu_convert_f32(F, F32)
            xq.zero_()
            return B.bicgstab_solve_f32prec(P, A, F32, rhs, x=xq, tol=tol, maxit=5000, work=sw)[1]

        def gmres20():
            B.bilu_factor(P, b, vals, F, fw)
            xg.zero_()
            return B.gmres_solve(P, A, F, rhs, x=xg, tol=tol, maxit=5000, restart=20, work=gw)[1]

        xp, xq, xg = torch.zeros_like(rhs), torch.zeros_like(rhs), torch.zeros_like(rhs)
        gw = B.workspace(int(B.L.load().gmres_workspace_bytes(P.handle, b, 20)), dev)
        row = {"workload": "grid96x96x48_7pt", "b": b, "k": k}
        for name, fn in (("fp64", fp64), ("mixed", mixed), ("f32prec", f32prec),
                         ("f32prec_from_fp64", f32prec_from_fp64), ("fp64_gmres20", gmres20)):
            fn()  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            si = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            row[name] = {"ms": round(e0.elapsed_time(e1), 2), "iters": si.iters, "true_relres": si.true_relres,
                         "status": si.status}
        ref = oracle_solution(S, k) if with_oracle else None
        for name, xv in (("fp64", x64), ("mixed", x32), ("f32prec", xp), ("f32prec_from_fp64", xq),
                         ("fp64_gmres20", xg)):
            if ref is not None:
                row[name]["x_rel_err_vs_oracle"] = rel_err(xv, ref["x"])
            if name != "fp64":
                row[name + "_speedup"] = round(row["fp64"]["ms"] / row[name]["ms"], 3)
        if ref is not None:
            row["oracle_reference"] = {k2: ref[k2] for k2 in ("iters", "true_relres", "status", "seconds")}
        out.append(row)
        P.close()
    return out


def fp32_kernel_rates(B, S, P, F, vals, rhs, rp, ci, dev, stream, reps=10):
    """FP32-stored apply and FP32 SpMV on the main workload: mean CUDA-event
    time and algorithmic GB/s (4-byte values).  spmv_f32 reads x in FP64,
    spmv_f32x in FP32 (the SpMV of the mixed solve, on the FP32 apply's
    result)."""
    import torch
    info = P.info
    b = S.b
    ab = algorithmic_bytes(S.n, b, S.nnzb, info.nnz_l, info.nnz_u, v=4)
    F32 = B.bilu_convert_f32(F)
    V32 = B.bilu_convert_f32(vals)
    aw = B.workspace(P.apply_workspace_bytes(b), dev)
    x, y = torch.empty_like(rhs), torch.empty_like(rhs)
    res = {}
    x32 = rhs.float()
    for name, fn, by in (("apply_f32", lambda: B.bilu_apply_f32(P, b, F32, rhs, x, aw), ab["apply"]),
                         ("spmv_f32", lambda: B.bsr_spmv_f32(S.n, b, rp, ci, V32, rhs, y), ab["spmv"]),
                         ("spmv_f32x", lambda: B.bsr_spmv_f32x(S.n, b, rp, ci, V32, x32, y),
                          ab["spmv"] - 4 * S.n * b)):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"avg_us": round(ms * 1e3, 1), "gbs": round(by / (ms * 1e-3) / 1e9, 1)}
    return res


def _oracle_ref_job(job):
    """Worker of the sweep's process pool (spawned, so it holds no CUDA
    context): the oracle's FP64 solution of one generated system."""
    wl, b, k = job
    from paper_1703_01325_gb300.reservoir import WORKLOADS, reservoir_system
    cfg = dict(WORKLOADS[wl])
    cfg["b"] = b
    ref = oracle_solution(reservoir_system(**cfg), k, tol=1e-10, maxit=2000)
    return job, ref


def sweep(B, dev, stream, which, tol=1e-8, reps=20, with_oracle=False, solve_reps=None, emit=True):
    """Per-configuration numbers, one JSON line each: the device set-up
    (symbolic phase and schedules, bilu_symbolic_gpu + bilu_pattern_upload),
    FP64 and FP32 factorization, FP64 and FP32 apply and SpMV (mean CUDA-event
    time over `reps` calls, algorithmic GB/s), and the solvers from x0 = 0
    toward a true relative residual of `tol`.

    c2 (96 x 96 x 48, b in {2,4,6,8}, k in {0,1,2}): BiCGSTAB with the FP64
    preconditioner and with the FP32-stored one (best of 3 solves,
    factorization excluded); with `with_oracle`, each solution's error against
    the CPU oracle's FP64 solution (computed by a pool of spawned processes on
    the host cores while the GPU sweeps) and the oracle's kernel times.

    c3 (160 x 160 x 80 27-point ILU(2)): no solver reaches 1e-8, so the four
    solvers get the same budget of work and report where they stand: FP64
    BiCGSTAB and FP32-preconditioned BiCGSTAB with 300 iterations (two applies
    and two SpMVs each), FP64 refinement around FP32 BiCGSTAB with 300 inner
    iterations, GMRES(20) with 600 Arnoldi steps (one apply and one SpMV
    each); also the host symbolic phase for comparison with the device one."""
    import torch
    from paper_1703_01325_gb300.reservoir import WORKLOADS, reservoir_system
    if which == "c2":
        cases = [("grid96x96x48_7pt", b, k) for b in (2, 4, 6, 8) for k in (0, 1, 2)]
        maxit, nrep = 5000, 3
    else:
        cases = [("grid160x160x80_27pt_b3", 3, 2)]
        maxit, nrep = 300, 1
    solve_reps = solve_reps or nrep
    hbm, _ = peaks()
    pool = refs = None
    if with_oracle and which == "c2":
        import multiprocessing as mp
        # a quarter of the host cores: the solves' host loop (a state read
        # every few iterations) must not wait for a core
        pool = mp.get_context("spawn").Pool(min(len(cases), max(1, (os.cpu_count() or 4) // 4)))
        refs = pool.map_async(_oracle_ref_job, cases)

    def timed(fn, n):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    def timed_solve(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        si = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms": round(e0.elapsed_time(e1), 2), "iters": si.iters, "true_relres": si.true_relres,
                "status": si.status}

    rows, xs, systems = [], {}, {}
    for wl, b, k in cases:
        if (wl, b) not in systems:  # the matrix does not depend on k
            systems.clear()
            cfg = dict(WORKLOADS[wl])
            cfg["b"] = b
            systems[(wl, b)] = reservoir_system(**cfg)
        S = systems[(wl, b)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P = B.bilu_symbolic_gpu(S.n, S.row_ptr, S.col_idx, k)
        t1 = time.perf_counter()
        P.upload()
        t2 = time.perf_counter()
        info = P.info
        rp, ci = torch.from_numpy(S.row_ptr).to(dev), torch.from_numpy(S.col_idx).to(dev)
        vals, rhs = torch.from_numpy(S.vals.reshape(-1)).to(dev), torch.from_numpy(S.rhs).to(dev)
        A = (S.n, b, rp, ci, vals)
        F = B.new_factors(P, b, dev)
        F32 = torch.empty(max(P.factor_bytes_f32(b) // 4, 1), dtype=torch.float32, device=dev)
        fw = B.workspace(P.factor_workspace_bytes(b), dev)
        aw = B.workspace(P.apply_workspace_bytes(b), dev)
        sw = B.workspace(P.bicgstab_workspace_bytes(b), dev)
        V32 = B.bilu_convert_f32(vals)
        x, y = torch.empty_like(rhs), torch.empty_like(rhs)
        row = {"workload": wl, "b": b, "k": k, "n": S.n, "nnzb": S.nnzb, "nnz_l": info.nnz_l,
               "nnz_u": info.nnz_u, "levels_lower": info.nlev_l,
               "setup_ms": {"symbolic_gpu": round((t1 - t0) * 1e3, 1), "schedules_upload": round((t2 - t1) * 1e3, 1),
                            "total": round((t2 - t0) * 1e3, 1)}}
        row["factor_ms"] = round(timed(lambda: B.bilu_factor(P, b, vals, F, fw), 3), 2)
        row["factor_f32_ms"] = round(timed(lambda: B.bilu_factor_f32(P, b, vals, F32, fw), 3), 2)
        B.bilu_factor(P, b, vals, F, fw)
        B.bilu_convert_f32(F, F32)
        for v, tag in ((8, "f64"), (4, "f32")):
            ab = algorithmic_bytes(S.n, b, S.nnzb, info.nnz_l, info.nnz_u, v=v)
            if tag == "f64":
                fa = lambda: B.bilu_apply(P, b, F, rhs, x, aw)
                fs = lambda: B.bsr_spmv(S.n, b, rp, ci, vals, rhs, y)
            else:
                fa = lambda: B.bilu_apply_f32(P, b, F32, rhs, x, aw)
                fs = lambda: B.bsr_spmv_f32(S.n, b, rp, ci, V32, rhs, y)
            kerns = [("apply", fa, ab["apply"]), ("spmv", fs, ab["spmv"])]
            if tag == "f32":  # the mixed solve's SpMV: x in FP32, as the FP32 apply leaves it
                x32 = rhs.float()
                kerns.append(("spmv_x32", lambda: B.bsr_spmv_f32x(S.n, b, rp, ci, V32, x32, y),
                              ab["spmv"] - 4 * S.n * b))
            for name, fn, by in kerns:
                ms = timed(fn, reps)
                gbs = by / (ms * 1e-3) / 1e9
                row[f"{name}_{tag}"] = {"us": round(ms * 1e3, 1), "gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm, 3)}
        if which == "c2":
            for tag, fac in (("bicgstab_f64", None), ("bicgstab_f32prec", F32)):
                runs = []
                for _ in range(solve_reps):
                    x.zero_()
                    if fac is None:
                        r = timed_solve(lambda: B.bicgstab_solve(P, A, F, rhs, x=x, tol=tol, maxit=maxit, work=sw)[1])
                    else:
                        r = timed_solve(lambda: B.bicgstab_solve_f32prec(P, A, F32, rhs, x=x, tol=tol, maxit=maxit,
                                                                         work=sw)[1])
                    runs.append(r)
                # best of the runs: host-side delays between the solver's
                # state reads only ever add time
                runs.sort(key=lambda r: r["ms"])
                row[tag] = dict(runs[0], runs=len(runs))
                if refs is not None:
                    xs[(b, k, tag)] = x.cpu().numpy()
            if with_oracle:
                row["cpu_baseline"] = oracle_kernel_times(S, k)
        else:
            mw = B.workspace(P.bicgstab_mixed_workspace_bytes(b), dev)
            gw = B.workspace(int(B.L.load().gmres_workspace_bytes(P.handle, b, 20)), dev)
            x.zero_()
            row["bicgstab_f64"] = timed_solve(lambda: B.bicgstab_solve(P, A, F, rhs, x=x, tol=tol, maxit=300,
                                                                       work=sw)[1])
            x.zero_()
            row["bicgstab_f32prec"] = timed_solve(lambda: B.bicgstab_solve_f32prec(P, A, F32, rhs, x=x, tol=tol,
                                                                                   maxit=300, work=sw)[1])
            x.zero_()
            row["mixed_refinement"] = timed_solve(lambda: B.bicgstab_solve_mixed(
                P, A, V32, F32, rhs, x=x, tol=tol, maxit=300, inner_tol=1e-3, inner_maxit=100, work=mw)[1])
            x.zero_()
            row["gmres20_f64"] = timed_solve(lambda: B.gmres_solve(P, A, F, rhs, x=x, tol=tol, maxit=600, restart=20,
                                                                   work=gw)[1])
            row["budget"] = ("equal work: 300 BiCGSTAB iterations (2 applies + 2 SpMVs each), 300 inner iterations of "
                             "the refinement, 600 GMRES(20) steps (1 apply + 1 SpMV each)")
            t3 = time.perf_counter()
            H = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, k)
            row["setup_ms"]["symbolic_host_for_comparison"] = round((time.perf_counter() - t3) * 1e3, 1)
            H.close()
            del mw, gw
        rows.append(row)
        if refs is None and emit:
            print(json.dumps(row), flush=True)
        del F, F32, fw, aw, sw, V32, vals
        P.close()
        torch.cuda.empty_cache()
    if refs is not None:
        import numpy as np
        done = dict(refs.get())
        pool.close()
        pool.join()
        for row in rows:
            ref = done[("grid96x96x48_7pt", row["b"], row["k"])]
            for tag in ("bicgstab_f64", "bicgstab_f32prec"):
                xv = xs[(row["b"], row["k"], tag)]
                row[tag]["x_rel_err_vs_oracle"] = float(np.linalg.norm(xv - ref["x"]) / np.linalg.norm(ref["x"]))
            row["oracle_reference"] = {k2: ref[k2] for k2 in ("iters", "true_relres", "status", "seconds")}
            if emit:
                print(json.dumps(row), flush=True)
    return rows


def c2_summary(rows):
    """The b x k sweep of the 96 x 96 x 48 grid in brief: per configuration
    the FP64 and FP32 apply and SpMV times and one FP64 and one
    FP32-preconditioned BiCGSTAB solve to 1e-8 (factorization excluded)."""
    out = []
    for r in rows:
        f64, f32 = r["bicgstab_f64"], r["bicgstab_f32prec"]
        out.append({"b": r["b"], "k": r["k"], "levels": r["levels_lower"],
                    "apply_us": {"f64": r["apply_f64"]["us"], "f32": r["apply_f32"]["us"]},
                    "apply_frac_hbm_f64": r["apply_f64"]["frac_hbm"],
                    "spmv_us": {"f64": r["spmv_f64"]["us"], "f32": r["spmv_f32"]["us"],
                                "f32_x32": r["spmv_x32_f32"]["us"]},
                    "bicgstab_f64": {"ms": f64["ms"], "iters": f64["iters"], "status": f64["status"]},
                    "bicgstab_f32prec": {"ms": f32["ms"], "iters": f32["iters"], "status": f32["status"]},
                    "f32prec_speedup": round(f64["ms"] / f32["ms"], 3) if f32["ms"] > 0 else None})
    return out


def kernel_case(args):
    """One kernel family on one workload, args.reps launches after set-up, and
    a one-line status: the target of single-kernel profiler captures."""
    import torch
    import paper_1703_01325_gb300.bilu as B
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    S, _ = system(args)
    b = S.b
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, args.k).upload()
    rp, ci = torch.from_numpy(S.row_ptr).to(dev), torch.from_numpy(S.col_idx).to(dev)
    vals, rhs = torch.from_numpy(S.vals.reshape(-1)).to(dev), torch.from_numpy(S.rhs).to(dev)
    F, _ = B.bilu_factor(P, b, vals)
    aw = B.workspace(P.apply_workspace_bytes(b), dev)
    x = torch.empty_like(rhs)
    if args.kernel_case == "apply":
        fn = lambda: B.bilu_apply(P, b, F, rhs, x, aw)
    elif args.kernel_case == "apply_f32":
        F32 = B.bilu_convert_f32(F)
        fn = lambda: B.bilu_apply_f32(P, b, F32, rhs, x, aw)
    elif args.kernel_case == "spmv":
        fn = lambda: B.bsr_spmv(S.n, b, rp, ci, vals, rhs, x)
    elif args.kernel_case == "spmv_f32":
        V32 = B.bilu_convert_f32(vals)
        fn = lambda: B.bsr_spmv_f32(S.n, b, rp, ci, V32, rhs, x)
    else:
        V32, x32 = B.bilu_convert_f32(vals), rhs.float()
        fn = lambda: B.bsr_spmv_f32x(S.n, b, rp, ci, V32, x32, x)
    for _ in range(args.reps):
        fn()
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "workload": args.workload, "b": b, "k": args.k,
                      "reps": args.reps, "workspace_status": B.bilu_workspace_status(aw)}))
    P.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.kernel_case:
        kernel_case(args)
        return
    if args.sweep:
        import torch
        import paper_1703_01325_gb300.bilu as B
        dev = torch.device("cuda:0")
        torch.cuda.set_device(dev)
        sweep(B, dev, torch.cuda.current_stream(dev), args.sweep, with_oracle=args.oracle)
        return
    import numpy as np
    import torch

    import paper_1703_01325_gb300.bilu as B
    from paper_1703_01325_gb300 import _lib as L

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist, world, rank, local = replica_group("nccl", torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    lib = L.load()
    if args.chunk:
        B.bilu_set_trisolve_chunk(args.chunk)

    S, cfg = system(args)
    b = S.b
    t0 = time.perf_counter()
    P = B.bilu_symbolic(S.n, S.row_ptr, S.col_idx, args.k)
    symbolic_ms = (time.perf_counter() - t0) * 1e3
    P.upload()
    info = P.info
    rp = torch.from_numpy(S.row_ptr).to(dev)
    ci = torch.from_numpy(S.col_idx).to(dev)
    vals = torch.from_numpy(S.vals.reshape(-1)).to(dev)
    rhs = torch.from_numpy(S.rhs).to(dev)
    F = B.new_factors(P, b, dev)
    fwork = B.workspace(P.factor_workspace_bytes(b), dev)
    swork = B.workspace(P.bicgstab_workspace_bytes(b), dev)
    x = torch.zeros_like(rhs)
    A = (S.n, b, rp, ci, vals)
    stream = torch.cuda.current_stream()

    def step():
        B.bilu_factor(P, b, vals, F, fwork)
        x.zero_()
        _, si = B.bicgstab_solve(P, A, F, rhs, x=x, tol=args.tol, maxit=args.maxit, work=swork)
        return si

    for _ in range(args.warmup):
        si = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    lib.bilu_profile_enable(1)
    launches0 = lib.bilu_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            si = step()
            iters.append((si.status, si.iters, si.true_relres))
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = lib.bilu_launch_count() - launches0
    prof = {}
    for kid, name in enumerate(L.PROF_KERNELS):
        nl, tm = C.c_int64(), C.c_double()
        lib.bilu_profile_read(kid, C.byref(nl), C.byref(tm))
        prof[name] = (nl.value, tm.value)
    lib.bilu_profile_enable(0)
    if dist:
        ms = max_over_ranks(ms, dist, dev)

    ab = algorithmic_bytes(S.n, b, S.nnzb, info.nnz_l, info.nnz_u)
    hbm, peak_src = peaks()
    kern = {}
    for name in ("spmv", "lower_solve", "diag_scale", "upper_solve"):
        nl, tm = prof[name]
        if nl:
            avg_ms = tm / nl
            kern[name] = {"launches": nl, "avg_us": round(avg_ms * 1e3, 2),
                          "gbs": round(ab[name] / (avg_ms * 1e-3) / 1e9, 1),
                          "share": round(tm / (ms * args.steps), 3)}
    top = max(kern, key=lambda k: kern[k]["share"]) if kern else None
    roof = None
    if top:
        ach = kern[top]["gbs"]
        traffic = NCU_TRAFFIC.get((args.workload, args.k, top))
        roof = {"kernel": top, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 3), "traffic": traffic, "peak_source": peak_src,
                "algorithmic_bytes": ab[top]}

    # end to end through the public API: pinned host A values and rhs in, x out
    e2e = None
    if not args.no_e2e:
        h_vals = torch.from_numpy(S.vals.reshape(-1)).pin_memory()
        h_rhs = torch.from_numpy(S.rhs).pin_memory()
        h_x = torch.empty_like(h_rhs).pin_memory()
        d_vals = torch.empty_like(vals)
        d_rhs = torch.empty_like(rhs)

        def e2e_step():
            d_vals.copy_(h_vals, non_blocking=True)
            d_rhs.copy_(h_rhs, non_blocking=True)
            B.bilu_factor(P, b, d_vals, F, fwork)
            x.zero_()
            B.bicgstab_solve(P, (S.n, b, rp, ci, d_vals), F, d_rhs, x=x, tol=args.tol, maxit=args.maxit,
                             work=swork)
            h_x.copy_(x, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        g1.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": round(g0.elapsed_time(g1) / args.steps, 3), "unit": "ms",
               "h2d_bytes_per_step": int(h_vals.numel() * 8 + h_rhs.numel() * 8),
               "d2h_bytes_per_step": int(h_x.numel() * 8)}

    small = prec = f32 = c2 = sweep_c2 = None
    if rank == 0 and args.workload == WORKLOAD and not args.no_extras:
        small = ms_to_tol_small(B, dev, stream)
        c2 = ms_to_tol_c2(B, dev, stream)
        f32 = fp32_kernel_rates(B, S, P, F, vals, rhs, rp, ci, dev, stream)
        if not args.no_precision:
            prec = precision_compare(B, dev, stream, with_oracle=not args.no_cpu)
        if not args.no_c2:
            # the b x k sweep in brief (one solve each, no oracle references;
            # `--sweep c2 --oracle` gives the full record); a failure here
            # must not cost the bench line
            try:
                sweep_c2 = {"workload": "grid96x96x48_7pt", "tol": 1e-8,
                            "rows": c2_summary(sweep(B, dev, stream, "c2", reps=5, solve_reps=1, emit=False))}
            except Exception as exc:  # noqa: BLE001
                sweep_c2 = {"error": f"{type(exc).__name__}: {exc}"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    statuses = sorted({s for s, _, _ in iters})
    gpu_iters = iters[-1][1]
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(S, args.k, gpu_iters)
    factor_ms = prof["backfill"][1] + prof["factor"][1] + prof["scale_upper"][1] + prof["factor_init"][1]
    clk = clocks.summary()
    ceil = None
    if kern:
        sm_mhz = clk.get("sm_mhz") or 2070.0
        ceil = fp64_issue_ceiling(P, b, torch.cuda.get_device_properties(dev).multi_processor_count, sm_mhz)
        for name in ("lower_solve", "upper_solve"):
            if name in kern:
                ceil[name]["measured_us"] = kern[name]["avg_us"]
                ceil[name]["frac"] = round(ceil[name]["ceiling_us"] / kern[name]["avg_us"], 3)
        ceil["note"] = ("FP64 issue bound of each FP64 sweep at the sampled SM clock: "
                        "ceil(blocks/G)*b DFMA + log2(G) DADD warp instructions per row, "
                        "one FP64 warp instruction per 19 cycles per SM; frac = ceiling / measured")
    if roof is not None and ceil is not None and roof["kernel"] in ceil:
        roof["fp64_issue_frac"] = ceil[roof["kernel"]]["frac"]
    out = {
        "metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "k": args.k, "tol": args.tol, "maxit": args.maxit, **cfg,
                   "n": S.n, "nnzb": S.nnzb, "nnz_p": info.nnz_p, "levels_lower": info.nlev_l,
                   "trisolve_chunk": B.bilu_get_trisolve_chunk() or "auto (two grid lines on natural-order grids)",
                   "l2": "inputs larger than L2 (A values %.0f MB, factors %.0f MB)" % (
                       S.nnzb * b * b * 8 / 1e6, P.factor_bytes(b) / 1e6),
                   "step": ("backfill + factor + BiCGSTAB from x0 = 0 toward tol, at most maxit iterations; "
                            "this workload does not reach 1e-8 (nor does the CPU oracle), so a step is a "
                            "fixed budget of maxit iterations: 'ms to 1e-8' is measured on the converging "
                            "96x96x48 workload (ms_to_tol_c2) and on 16x16x8 (ms_to_tol_small)")},
        "converged": statuses == [0], "solve_status": statuses, "iters": gpu_iters,
        "true_relres": iters[-1][2],
        "factor_ms": round(factor_ms / args.steps, 3), "symbolic_ms": round(symbolic_ms, 1),
        "per_iteration_ms": round((ms - factor_ms / args.steps) / max(gpu_iters, 1), 4),
        "ms_to_tol_small": small, "ms_to_tol_c2": c2, "fp64_issue": ceil,
        "fp32_prec_vs_fp64": prec, "fp32_kernels": f32, "sweep_c2": sweep_c2,
        "kernels": kern, "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
        "gpu_launches": int(launches), "clocks": clk,
        "fp64_alu": {"peak_tflops": FP64_PEAK_TFLOPS,
                     "spmv_tflops": round(2 * S.nnzb * b * b / (kern["spmv"]["avg_us"] * 1e-6) / 1e12, 3)
                     if "spmv" in kern else None},
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
