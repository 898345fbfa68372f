#!/usr/bin/env python
"""Benchmark of the CP-GN hot path on one GB300 (replicas on N GPUs).

Workload (the configuration the headline metric is quoted on): a dense
order-3 400 x 400 x 400 FP32 tensor built from rank-50 N(0,1) factors with
column collinearity 0.9 plus 1e-6 relative Gaussian noise, decomposed at
rank R = 50 from a seeded N(0,1) starting point.  One step = one complete
CP-GN solve (Algorithm 1 with CP-CG, Algorithm 2) from that starting point to
relative stationarity sum||G||/sum||M|| <= 1e-8 with an FP64 gradient: the
mixed path forms every gradient as -E_(n) P^(n) from the residual tensor
E = X - [[A]] (reconstruction by error-free bf16 slice products on the
tcgen05 tensor cores, then the tcgen05 bf16x3 MTTKRP of E) and runs CP-CG
with FP32 vectors and FP64 scalars.  The value is the time to target
(seconds, lower is better); the same solve on the plain FP64 GPU path and the
all-mode MTTKRP throughput are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own replica; rank 0 prints one
JSON line with the maximum time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CP-GN time-to-residual 1e-8 and all-mode MTTKRP TFLOP/s vs plain FP64 GPU path"
WORKLOAD = "collinear400"
WORKLOAD_DESC = ("400x400x400 FP32 tensor, rank-50 N(0,1) factors with column collinearity 0.9, "
                 "1e-6 relative noise; R=50; seeded N(0,1) start")
TARGET_STAT = 1e-8
# The metric's name says "residual 1e-8"; on FP32-stored inputs with 1e-6 noise the relative residual
# cannot fall below ~1e-6, so the solve is timed to relative stationarity instead (Algorithm 1's loop
# test on sum||G||, made scale-free), with an FP64-accurate gradient.
TARGET_NOTE = ("time to relative stationarity sum||G||/sum||M|| <= 1e-8 (FP64-accurate gradient) in place of "
               "residual 1e-8, which FP32 storage and the 1e-6 noise floor make unreachable")
CONFIG = {"workload": f"{WORKLOAD}: {WORKLOAD_DESC}",
          "target": f"sum||G||/sum||M|| <= {TARGET_STAT} with an FP64 gradient",
          "target_note": TARGET_NOTE,
          "step": "one full CP-GN solve (residual-form gradient every iteration, FP32 CG vectors)",
          "l2": "inputs larger than L2 (X 256 MB, planes of E 256 MB)"}
MAX_GN = 300
EPS_CG = 1e-3
CG_MAX = 250
MU = 2.0
# DRAM traffic of the dominant kernels from one ncu capture each (profiles/pcg_kernel_collinear400.md,
# profiles/resid_gradient_collinear400.md).  It is reported only while every source of the record
# still has the SHA-1 it had when the counters were taken.
PROFILED = {
    "pcg": {"src": {"paper_1910_12331_gb300/csrc/k_pcg.cu": "8d1f61e031a45b4987413092a51efb5b5ab5c16b",
                    "paper_1910_12331_gb300/csrc/common.cuh": "40734fb1244aa169472e951051e1c496044bcc11"},
            "dram_bytes": 966656 + 136960, "cg_iters": 27},
    # recon_tc_kernel (272687360 B read + 244927232 B written) + mttkrp_tc_kernel (391966464 + 7487488)
    "gradient": {"src": {"paper_1910_12331_gb300/csrc/k_resid_tc.cu": "e1d375b16ea4885322925fd0296c72138322ddbb",
                         "paper_1910_12331_gb300/csrc/k_mttkrp_tc.cu": "07a08367384d5c9fe3585da614836548472bec1a"},
                 "dram_bytes": 272687360 + 244927232 + 391966464 + 7487488},
}
# The mixed path of the timed solve: residual-form gradient every iteration, FP32 CG vectors.
MIXED = {"prec": "residual", "cg_fp32": True}


def profiled(key):
    """The profiled record of a kernel if its source is unchanged since the capture, else None."""
    import hashlib

    rec = PROFILED[key]
    for src, sha in rec["src"].items():
        try:
            digest = hashlib.sha1(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
        except OSError:
            return None
        if sha != digest:
            return None
    return rec


def lam_thresholds(A):
    """lambda_hi = 0.1 tau, lambda_lo = 1e-7 tau, tau = mean_n trace(Gamma^(n,n)) / R
    at the starting point (this project's convention for the thresholds of the
    varying rule; the paper gives no values)."""
    S = [a.T @ a for a in A]
    N, R = len(A), A[0].shape[1]
    traces = []
    for n in range(N):
        G = np.ones((R, R))
        for m in range(N):
            if m != n:
                G = G * S[m]
        traces.append(np.trace(G))
    tau = float(np.mean(traces)) / R
    return 0.1 * tau, 1e-7 * tau


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, pg, device):
    """The largest value over the ranks of the process group (the job's time is
    the slowest replica's), or the value itself without a group."""
    if pg is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--id={self.index}",
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self._proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def wait_first(self, timeout_s=5.0):
        """Block until nvidia-smi has produced its first sample (its start-up
        then lies outside any region timed afterwards)."""
        t0 = time.time()
        while self._proc and not self.samples and time.time() - t0 < timeout_s:
            time.sleep(0.01)

    def mark(self):
        return len(self.samples)

    def __exit__(self, *exc):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self, i0=0, i1=None):
        """Clock median and throttle reasons over samples [i0, i1] (the timed region
        and the sample taken right after it)."""
        sel = self.samples[i0:(None if i1 is None else i1 + 1)] or self.samples[-1:]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in sel if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in sel if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in sel:
            for k, nm in enumerate(names):
                if len(s) > 4 + k and s[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sel)}


def oracle_solve(p, lam_hi, lam_lo):
    """The FP64 oracle (as it stands) solving the workload to the same target
    as the GPU: Algorithm 1 with CP-CG to eps_cg = 1e-3, dimension-tree
    MTTKRP, the same lambda schedule and starting point.  Returns (seconds,
    info, cores)."""
    import oracle

    oracle.build()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    _, st, info = oracle.gn_solve(p["X"], [a.copy() for a in p["init"]], lam_hi, lam_lo, lam_hi, MU, EPS_CG,
                                  CG_MAX, TARGET_STAT, MAX_GN)
    return time.perf_counter() - t0, dict(info, status=st), cores


def oracle_gn_iteration(p, lam_hi, lam_lo, threads):
    """One GN iteration of the oracle from the starting point on `threads`
    threads (seconds)."""
    import oracle

    oracle.build()
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.gn_step(p["X"], [a.copy() for a in p["init"]], lam_hi, 0, lam_lo, lam_hi, MU, EPS_CG, CG_MAX, 0, True)
    dt = time.perf_counter() - t0
    oracle.set_threads(int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)))
    return dt


def cpu_baseline_record(p, lam_hi, lam_lo):
    """The oracle's full solve on all host cores (measured), plus the one-core
    figure: one GN iteration on one thread against one on all of them, which
    scales the measured full solve (a projection, marked as such)."""
    t_all, info, cores = oracle_solve(p, lam_hi, lam_lo)
    it1 = oracle_gn_iteration(p, lam_hi, lam_lo, 1)
    itn = oracle_gn_iteration(p, lam_hi, lam_lo, cores)
    return {"value": t_all, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": (f"one full FP64 oracle solve of the workload to the same target, timed once: "
                       f"{info['updates']} GN and {info['cg_iters']} CG iterations, stationarity "
                       f"{info['stationarity']:.3g}, converged={info['converged']}"),
            "one_core": {"value": t_all * it1 / itn, "unit": "s", "cores": 1,
                         "kind": "projected: measured solve x (one GN iteration on 1 thread / on all threads)",
                         "gn_iteration_s_1_core": it1, "gn_iteration_s_all_cores": itn}}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload(WORKLOAD, seed=0)
    lam_hi, lam_lo = lam_thresholds(p["init"])
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # warm-up: one GN iteration each (pages in the oracle and the workload; a solve keeps no other state)
    for _ in range(args.warmup):
        oracle_gn_iteration(p, lam_hi, lam_lo, cores)
    vals, info = [], None
    for _ in range(args.steps):
        t, info, cores = oracle_solve(p, lam_hi, lam_lo)
        vals.append(t)
    value = statistics.median(vals)
    sample = (f"each timed step is one full FP64 oracle solve of the workload to the target ({info['updates']} GN, "
              f"{info['cg_iters']} CG iterations); each warm-up step one GN iteration")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, parallelism=f"replicas x{args.gpus}"),
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cp_loss_timing(dev, reps=5):
    """Forward + backward of the CP loss ||X - [[A,B,C]]||^2 on the loss256
    workload (256^3 FP32, R=32 N(0,1) factors): the library's autograd
    Function (direct FP64 forward, fused all-mode MTTKRP backward) against
    torch.einsum autograd of the same loss in FP64."""
    import torch

    from paper_1910_12331_gb300 import autograd, datagen

    p = datagen.workload("loss256", seed=0)
    X = torch.from_numpy(p["X"]).to(dev)
    A0 = [torch.from_numpy(a.copy()).to(dev) for a in p["init"]]
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def ours(prec):
        A = [a.clone().requires_grad_() for a in A0]
        autograd.cp_loss(X, A, prec=prec).backward()

    def einsum():
        A = [a.clone().requires_grad_() for a in A0]
        ((X.double() - torch.einsum("iz,jz,kz->ijk", *A)) ** 2).sum().backward()

    return {"workload": "loss256: 256x256x256 FP32, R=32, N(0,1) factors", "unit": "ms (forward+backward)",
            "ours_bf16x3_backward": timed(lambda: ours("bf16x3")), "ours_fp64_backward": timed(lambda: ours("fp64")),
            "torch_einsum_fp64": timed(einsum)}


def batched_timing(dev, count=512):
    """The batched workload: 512 independent order-3 FP32 problems, sides
    uniform in 16..96, ranks uniform in 4..24, N(0,1) factors plus 1e-8
    relative noise, each solved to r <= 1e-6 (or 200 GN iterations) by one
    persistent kernel launch.  A plan is created once (the autotuner picks
    the block size on a scratch copy of the factors); the timed call is one
    plan launch captured in a CUDA graph and replayed, plus the result copy."""
    import torch

    from paper_1910_12331_gb300 import api, datagen

    probs = datagen.batched_problems(count, seed=0)
    Xs = [torch.from_numpy(p["X"]).to(dev) for p in probs]
    h = api.Handle(dev)
    stream = torch.cuda.current_stream(dev)
    b = []
    for p, X in zip(probs, Xs):
        hi, lo = lam_thresholds(p["init"])
        b.append(dict(X=X, A=[torch.from_numpy(a.copy()).to(dev) for a in p["init"]], lam=hi, lam_lo=lo,
                      lam_hi=hi, mu=MU))
    init = [[a.clone() for a in q["A"]] for q in b]
    t0 = time.perf_counter()
    plan = api.BatchPlan(h, b, EPS_CG, CG_MAX, 200, 1e-6, autotune=True)
    tune_s = time.perf_counter() - t0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.launch()
    for q, a0 in zip(b, init):
        for a, c in zip(q["A"], a0):
            a.copy_(c)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.replay()
    res = plan.results()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    threads, order = plan.threads, plan.order
    plan.close()
    conv = sum(r["converged"] for r in res)
    # the same batch with step-size control by Armijo's condition (one-shot call, untimed beside the graph)
    b_ls = []
    for q, a0 in zip(b, init):
        q2 = dict(q, A=[a.clone() for a in a0], armijo_c=1e-4, armijo_beta=0.5, armijo_max=10)
        b_ls.append(q2)
    t1 = time.perf_counter()
    res_ls = api.cp_gn_solve_batched(h, b_ls, EPS_CG, CG_MAX, 200, 1e-6)
    t_ls = time.perf_counter() - t1
    armijo = {"converged": sum(r["converged"] for r in res_ls), "wall_s": t_ls,
              "gn_iters_mean": float(np.mean([r["iters"] for r in res_ls])),
              "backtracks": sum(r["ls_backtracks"] for r in res_ls),
              "status_counts": {str(k): sum(1 for r in res_ls if r["status"] == k)
                                for k in sorted({r["status"] for r in res_ls})},
              "not_converged": [{"problem": i, "status": r["status"], "iters": r["iters"],
                                 "rel_residual": r["rel_residual"]} for i, r in enumerate(res_ls) if not r["converged"]]}
    h.close()
    # Algorithmic work of the timed solve, per problem (order 3, Pi = s1 s2 s3, S = s1 + s2 + s3): per GN
    # iteration 6 Pi R flops (the all-mode MTTKRP by the dimension tree, 4 Pi R, and the stop test's
    # reconstruction, 2 Pi R) plus 6 S R^2 (Grams, gradient, update); per CG iteration 16 S R^2 (the implicit
    # matvec's three R x R products per row and the preconditioner's one).  Against the FP32 FMA peak of the
    # GPU at 2070 MHz (SMs x 128 lanes x 2 flops): the kernel runs this arithmetic in FP32 on the CUDA cores.
    work = []
    for p, r in zip(probs, res):
        d3, R = p["X"].shape, p["truth"][0].shape[1]
        Pi, S = float(np.prod(d3)), float(sum(d3))
        work.append(r["iters"] * (6.0 * Pi * R + 6.0 * S * R * R) + r["cg_iters_total"] * 16.0 * S * R * R)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * 2.07e9 / 1e12
    achieved = float(np.sum(work)) / (ms / 1e3) / 1e12
    imax = int(np.argmax(work))
    roof = {"bound": "latency (one CTA per problem, every step a block-level reduction)", "gflop": float(np.sum(work)) / 1e9,
            "achieved_tflops": achieved, "fp32_peak_tflops": fp32_peak, "frac": achieved / fp32_peak,
            "largest_problem": {"problem": imax, "gflop": work[imax] / 1e9, "gn_iters": res[imax]["iters"],
                                "cg_iters": res[imax]["cg_iters_total"], "share_of_work": work[imax] / float(np.sum(work))}}
    return {"workload": f"{count} order-3 FP32 problems, sides U{{16..96}}, ranks U{{4..24}}, N(0,1) factors, "
                        "1e-8 noise; target r <= 1e-6 or 200 GN iterations",
            "ms": ms, "problems_per_s": count / (ms / 1e3), "converged": conv, "roofline": roof,
            "gn_iters_mean": float(np.mean([r["iters"] for r in res])),
            "cg_iters_mean": float(np.mean([r["cg_iters_total"] for r in res])),
            "cg_breakdowns": sum(r["cg_breakdowns"] for r in res),
            "status_counts": {str(k): sum(1 for r in res if r["status"] == k) for k in sorted({r["status"] for r in res})},
            # without step-size control a GN step can overshoot; a problem whose factors then grow until a
            # pivot of the preconditioner's factorisation is no longer positive ends with CP_ERR_NOT_SPD (5)
            "not_converged": [{"problem": i, "status": r["status"], "iters": r["iters"],
                               "rel_residual": r["rel_residual"]} for i, r in enumerate(res) if not r["converged"]],
            "launches": 1, "graph": "one captured plan launch, replayed", "threads_per_cta": threads,
            "problem_order": ["given", "largest work first"][order], "autotune_s": tune_s,
            "with_armijo": armijo}


def c1_timing(dev, seeds=range(10)):
    """The exact 20^3 rank-5 Gaussian tensors (FP64, no noise), seeds 0..9: time
    to r <= 1e-10 from the seeded N(0,1) start, Gauss-Newton (Algorithm 1, FP64)
    and ALS (Section 2.2, FP64), on the GPU through the C ABI, and the FP64
    oracle on the host cores doing the same."""
    import torch

    import oracle
    from paper_1910_12331_gb300 import api, datagen

    h = api.Handle(dev)
    out = {"gn": [], "als": [], "oracle_gn": [], "oracle_als": []}
    for seed in seeds:
        p = datagen.workload("exact20", seed=seed)
        hi, lo = lam_thresholds(p["init"])
        X = torch.from_numpy(p["X"]).to(dev)
        A = [torch.from_numpy(a.copy()).to(dev) for a in p["init"]]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, res = api.cp_gn_solve(h, X, A, api.gn_params(hi, lo, hi, MU, EPS_CG, CG_MAX),
                                 api.solve_opts(max_iters=100, target_residual=1e-10))
        out["gn"].append((time.perf_counter() - t0, res["iters"], bool(res["converged"])))
        A = [torch.from_numpy(a.copy()).to(dev) for a in p["init"]]
        t0 = time.perf_counter()
        it, r = 0, 1.0
        while it < 1000 and r > 1e-10:
            r = api.cp_als_sweep(h, X, A, 0.0, "fp64")
            it += 1
        out["als"].append((time.perf_counter() - t0, it, r <= 1e-10))
        # the oracle on the host cores (baseline)
        Ao, lam, d = [a.copy() for a in p["init"]], hi, 0
        t0 = time.perf_counter()
        it, r = 0, 1.0
        while it < 100 and r > 1e-10:
            Ao, lam, d, _, _ = oracle.gn_step(p["X"], Ao, lam, d, lo, hi, MU, EPS_CG, CG_MAX)
            r = oracle.residual(p["X"], Ao)
            it += 1
        out["oracle_gn"].append((time.perf_counter() - t0, it, r <= 1e-10))
        Ao = [a.copy() for a in p["init"]]
        t0 = time.perf_counter()
        it, r = 0, 1.0
        while it < 1000 and r > 1e-10:
            Ao, _ = oracle.als_sweep(p["X"], Ao)
            r = oracle.residual(p["X"], Ao)
            it += 1
        out["oracle_als"].append((time.perf_counter() - t0, it, r <= 1e-10))
    h.close()

    def summ(v):
        return {"median_s": statistics.median(x[0] for x in v), "iters": [x[1] for x in v],
                "converged": sum(x[2] for x in v)}

    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"workload": "exact20: 20x20x20 FP64 = [[A*]], rank-5 N(0,1) factors, no noise; R=5; seeds 0..9",
            "target": "relative residual <= 1e-10", "unit": "s (wall time per solve, median over seeds)",
            "gn": summ(out["gn"]), "als": summ(out["als"]),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "gn": summ(out["oracle_gn"]),
                             "als": summ(out["oracle_als"]), "sample": "the same ten solves on the host cores"}}


def c3_timing(dev, max_gn=60, max_als=400):
    """The order-4 120^4 FP32 workload (rank-40 U(0,1) factors, 1e-4 noise; R=40):
    Gauss-Newton (mixed path: residual-form gradient, FP32 CG vectors) against
    ALS (bf16x3 tensor-core MTTKRP mode by mode), both from the seeded start, to
    the relative residual 1.00001 r(A*) (A* the generating factors, so the
    optimum lies below it), the residual evaluated after every iteration by the
    tensor-core reconstruction (cp_residual_tensor, sums only)."""
    import torch

    from paper_1910_12331_gb300 import api, datagen

    p = datagen.workload("uniform120x4", seed=0)
    X = torch.from_numpy(p["X"]).to(dev)
    h = api.Handle(dev)

    def resid(A):
        _, e, x = api.cp_residual_tensor(h, X, A, sums_only=True)
        return float(np.sqrt(e / x))

    target = 1.00001 * resid([torch.from_numpy(a).to(dev) for a in p["truth"]])
    hi, lo = lam_thresholds(p["init"])
    runs = {}
    for method in ("gn", "als"):
        A = [torch.from_numpy(a.copy()).to(dev) for a in p["init"]]
        h.bump_version(X)
        params = api.gn_params(hi, lo, hi, MU, EPS_CG, CG_MAX, prec="residual", cg_fp32=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, r, cg = 0, 1.0, 0
        while r > target and it < (max_gn if method == "gn" else max_als):
            if method == "gn":
                _, st = api.cp_gn_step(h, X, A, params)
                cg += st["cg_iters"]
            else:
                api.cp_als_sweep(h, X, A, 0.0, "bf16x3", want_residual=False)
            r = resid(A)
            it += 1
        torch.cuda.synchronize()
        runs[method] = {"time_s": time.perf_counter() - t0, "iters": it, "rel_residual": r,
                        "converged": r <= target, **({"cg_iters": cg} if method == "gn" else {})}
    h.close()
    return {"workload": "uniform120x4: 120x120x120x120 FP32, rank-40 U(0,1) factors, 1e-4 relative noise; R=40",
            "target": f"relative residual <= 1.00001 r(A*) = {target:.6g}", "gn": runs["gn"], "als": runs["als"],
            "gn_speedup_over_als": runs["als"]["time_s"] / runs["gn"]["time_s"]}


def c3_cpu_sample():
    """One GN iteration and one ALS sweep of the FP64 oracle on the order-4
    workload, timed on the host cores (bounded sample; unit: s per iteration)."""
    import oracle
    from paper_1910_12331_gb300 import datagen

    p = datagen.workload("uniform120x4", seed=0)
    hi, lo = lam_thresholds(p["init"])
    t0 = time.perf_counter()
    oracle.gn_step(p["X"], [a.copy() for a in p["init"]], hi, 0, lo, hi, MU, EPS_CG, CG_MAX, 0, True)
    t_gn = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.als_sweep(p["X"], [a.copy() for a in p["init"]])
    t_als = time.perf_counter() - t0
    return {"kind": "oracle", "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "unit": "s per iteration", "gn_iteration_s": t_gn, "als_sweep_s": t_als,
            "sample": "one GN iteration (dimension-tree MTTKRP, CG to 1e-3) and one ALS sweep from the start"}


def exact_cp_cpu_sample():
    """One GN iteration (varying identity damping, from the start) of the FP64 oracle on each exact-CP
    workload with R above the sides, timed on the host cores (bounded sample; unit: s per iteration)."""
    import oracle
    from paper_1910_12331_gb300 import datagen

    out = {"kind": "oracle", "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
           "unit": "s per GN iteration", "sample": "one GN iteration (CG to 1e-3) from the start of each workload"}
    for name, sd, R, dist in (("gauss80_r120", 80, 120, "normal"), ("uniform11_150_r200", 150, 200, "uniform11")):
        p = datagen.make_problem((sd, sd, sd), R, dist=dist, dtype=np.float64, seed=0)
        hi, lo = lam_thresholds(p["init"])
        t0 = time.perf_counter()
        _, _, _, st, _ = oracle.gn_step(p["X"], [a.copy() for a in p["init"]], hi, 0, lo, hi, MU, EPS_CG, CG_MAX, 0,
                                        True)
        out[name] = {"gn_iteration_s": time.perf_counter() - t0, "cg_iters": st["cg_iters"]}
    return out


def likelihood_study(dev, n_problems=100, starts=15):
    """Section 5's convergence-likelihood study: for R = 3..9, n_problems exact
    rank-R 4x4x4 tensors from U(-1,1) factors, `starts` U(-1,1) starting points
    each; Gauss-Newton with the varying lambda run to r < 5e-5 or 500
    iterations, all problems in one batched launch.  Reported per rank: the
    problems with a converged start among the first 5 and among all starts
    (the paper's 5- and 15-initialisation curves)."""
    import torch

    from paper_1910_12331_gb300 import api, datagen

    probs = datagen.likelihood_problems(n_problems, range(3, 10), starts, 4, "uniform11", seed=0)
    h = api.Handle(dev)
    Xs = {}
    batch = []
    for q in probs:
        key = (q["rank"], q["problem"])
        if key not in Xs:
            Xs[key] = torch.from_numpy(q["X"]).to(dev)
        hi, lo = lam_thresholds(q["init"])
        batch.append(dict(X=Xs[key], A=[torch.from_numpy(a.copy()).to(dev) for a in q["init"]], lam=hi,
                          lam_lo=lo, lam_hi=hi, mu=MU))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = api.cp_gn_solve_batched(h, batch, EPS_CG, CG_MAX, 500, 5e-5)
    wall = time.perf_counter() - t0
    h.close()
    per_rank = {}
    for q, r in zip(probs, res):
        d = per_rank.setdefault(q["rank"], {})
        d.setdefault(q["problem"], []).append(bool(r["converged"]))
    table = {str(R): {"problems_with_a_converged_start_of_5": sum(any(v[:5]) for v in d.values()),
                      f"problems_with_a_converged_start_of_{starts}": sum(any(v) for v in d.values()),
                      "mean_converged_starts": float(np.mean([sum(v) for v in d.values()]))}
             for R, d in sorted(per_rank.items())}
    return {"workload": f"{n_problems} exact rank-R 4x4x4 tensors per R = 3..9, U(-1,1) factors, {starts} U(-1,1) "
                        "starts each; GN with varying lambda to r < 5e-5 or 500 iterations",
            "problems": len(probs), "wall_s": wall, "launches": 1, "per_rank": table}


def matmul_study(dev, inits=30):
    """Section 5's matrix-multiplication tensor: the 2x2 product tensor (4x4x4,
    rank 7), `inits` N(0,1) starts; ALS with lambda = 0.01 for 200 sweeps, then
    Gauss-Newton with the constant lambda = 1e-3, with and without Armijo's
    condition, to r <= 1e-8 or 300 iterations (FP64 path)."""
    import torch

    from paper_1910_12331_gb300 import api, datagen

    T = datagen.matmul_tensor(2)
    X = torch.from_numpy(T).to(dev)
    h = api.Handle(dev)
    rng = np.random.default_rng(0)
    out = {"armijo": 0, "plain": 0}
    t0 = time.perf_counter()
    for k in range(inits):
        A0 = [rng.standard_normal((4, 7)) for _ in range(3)]
        A = [torch.from_numpy(a).to(dev) for a in A0]
        for _ in range(200):
            api.cp_als_sweep(h, X, A, 0.01, "fp64", want_residual=False)
        warm = [a.clone() for a in A]
        for name, c in (("armijo", 1e-4), ("plain", 0.0)):
            B = [a.clone() for a in warm]
            params = api.gn_params(1e-3, 1e-3, 1e-3, MU, EPS_CG, CG_MAX, lam_fixed=True, armijo_c=c)
            _, res = api.cp_gn_solve(h, X, B, params, api.solve_opts(max_iters=300, target_residual=1e-8),
                                     check=False)
            out[name] += int(res["converged"] == 1)
    wall = time.perf_counter() - t0
    h.close()
    return {"workload": "2x2 matrix-multiplication tensor (4x4x4), rank 7; N(0,1) starts; 200 ALS sweeps at "
                        "lambda = 0.01, then GN at constant lambda = 1e-3", "inits": inits,
            "converged_gn_armijo": out["armijo"], "converged_gn_plain": out["plain"], "wall_s": wall}


def large_r_mttkrp(dev, reps=3):
    """The large-rank MTTKRP regime of Section 5 (s = R = 500, the exact-CP
    study; s = R = 800, the parallel-performance study): all-mode bf16x3 MTTKRP
    of U(0,1) FP32 tensors at rank R = s, where the contraction is
    compute-bound (R flop per byte of X); useful flops 4 prod(s) R per call."""
    import torch

    from paper_1910_12331_gb300 import api

    out = {}
    h = api.Handle(dev)
    for s_ in (500, 800):
        g = torch.Generator(device=dev).manual_seed(s_)
        X = torch.rand((s_, s_, s_), generator=g, device=dev, dtype=torch.float32)
        A = [torch.rand((s_, s_), generator=g, device=dev, dtype=torch.float64) for _ in range(3)]
        M = [torch.empty_like(a) for a in A]
        api.cp_mttkrp_all(h, X, A, M, prec="bf16x3")  # split of X cached, workspace grown
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            api.cp_mttkrp_all(h, X, A, M, prec="bf16x3")
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        flops = 4.0 * s_ ** 3 * s_
        out[f"s=R={s_}"] = {"ms": t * 1e3, "tflops_useful": flops / t / 1e12, "rank_tiles": (s_ + 63) // 64,
                            "x_bytes": 4 * s_ ** 3}
        del X, A, M
        torch.cuda.empty_cache()
    h.close()
    return {"workload": "U(0,1) FP32 s x s x s tensors, rank R = s; all-mode MTTKRP (bf16x3, tensor cores)",
            **out}


def exact_cp_study(dev, cap_s=6.0):
    """Section 5's sequential exact CP decompositions with the rank above the sides: s = 80, R = 120 with
    N(0,1) factors and s = 150, R = 200 with U(-1,1) factors (FP64 tensors of exact rank R, seeded starts
    from the same distribution).  Gauss-Newton with varying identity and varying diagonal damping (plain
    FP64 path; the CG kernel keeps its R x R matrices in global memory at these ranks) against FP64 ALS,
    each run until r <= 1e-10 or cap_s seconds; reported: the time at which r first fell below each
    decade and the final r."""
    import torch

    from paper_1910_12331_gb300 import api, datagen

    out = {"target": "relative residual <= 1e-10, or %.0f s" % cap_s}
    for name, s, R, dist in (("gauss80_r120", 80, 120, "normal"), ("uniform11_150_r200", 150, 200, "uniform11")):
        p = datagen.make_problem((s, s, s), R, dist=dist, dtype=np.float64, seed=0)
        X = torch.from_numpy(p["X"]).to(dev)
        h = api.Handle(dev)
        runs = {}
        for method in ("gn_identity", "gn_diag", "als"):
            A = [torch.from_numpy(a.copy()).to(dev) for a in p["init"]]
            hi, lo = lam_thresholds(p["init"])
            if method == "gn_diag":
                params = api.gn_params(0.1, 1e-7, 0.1, MU, EPS_CG, CG_MAX, prec="fp64", reg="diag")
            else:
                params = api.gn_params(hi, lo, hi, MU, EPS_CG, CG_MAX, prec="fp64")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, cg, r, marks = 0, 0, 1.0, {}
            while r > 1e-10 and time.perf_counter() - t0 < cap_s:
                if method == "als":
                    api.cp_als_sweep(h, X, A, 0.0, "fp64", want_residual=False)
                else:
                    st_code, st = api.cp_gn_step(h, X, A, params, check=False)
                    cg += st["cg_iters"]
                    if st_code not in (api.CP_OK, api.CP_WARN_CG_MAXIT):
                        break
                r = api.cp_residual(h, X, A)
                it += 1
                for d in range(1, 11):
                    key = "1e-%d" % d
                    if r <= 10.0 ** -d and key not in marks:
                        marks[key] = round(time.perf_counter() - t0, 4)
            runs[method] = {"iters": it, "final_r": r, "wall_s": time.perf_counter() - t0, "time_to_r": marks,
                            **({"cg_iters": cg} if method != "als" else {})}
        h.close()
        out[name] = {"workload": f"{s}x{s}x{s} FP64 = [[A*]], rank {R}, {dist} factors; R={R}", **runs}
        del X
    return out


def tucker_study(dev, direct_A):
    """Tucker compression ahead of CP (Section 1; Section 3.5's complexity comparison assumes it) on the
    timed workload: the truncated HoSVD of X to its multilinear rank (R, R, R), the GN solve of the R^3
    core (plain FP64 path, from the workload's start projected on the bases, B_n = U_n^T A0_n, formed on
    the host outside the timed parts, to the same stationarity target on the core), and A_n = U_n B_n;
    the relative residual of the expanded model against the direct solve's (direct_A)."""
    import torch

    from paper_1910_12331_gb300 import api, datagen

    p = datagen.workload(WORKLOAD, seed=0)
    X = torch.from_numpy(p["X"]).to(dev)
    R = p["init"][0].shape[1]
    ranks = (R,) * X.dim()
    h = api.Handle(dev)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    api.cp_hosvd(h, X, ranks)  # first call: module loads and workspace growth
    torch.cuda.synchronize()
    ev[0].record(stream)
    U, core, hos_it = api.cp_hosvd(h, X, ranks)
    ev[1].record(stream)
    torch.cuda.synchronize()
    B0 = [u.cpu().numpy().T @ a for u, a in zip(U, p["init"])]
    hi, lo = lam_thresholds(B0)
    B = [torch.from_numpy(np.ascontiguousarray(b)).to(dev) for b in B0]
    params = api.gn_params(hi, lo, hi, MU, EPS_CG, CG_MAX, prec="fp64")
    torch.cuda.synchronize()
    ev[2].record(stream)
    _, res = api.cp_gn_solve(h, core, B, params, api.solve_opts(max_iters=MAX_GN, target_stationarity=TARGET_STAT))
    ev[3].record(stream)
    A = api.cp_tucker_expand(h, U, B)
    ev[4].record(stream)
    torch.cuda.synchronize()
    e_full, x2 = api.cp_residual_sums(h, X, A)
    e_dir, _ = api.cp_residual_sums(h, X, direct_A)
    g2 = float(torch.sum(core * core))
    h.close()
    t_h, t_s, t_e = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3]), ev[3].elapsed_time(ev[4])
    return {"workload": f"{WORKLOAD}, compressed to its multilinear rank {ranks}",
            "hosvd_ms": t_h, "hosvd_iterations": hos_it,
            "core_solve_ms": t_s, "core_gn_iters": res["iters"],
            "core_cg_iters": res["cg_iters_total"], "core_converged": bool(res["converged"]),
            "expand_ms": t_e, "total_ms": t_h + t_s + t_e,
            "compression_rel_error": float(np.sqrt(max(x2 - g2, 0.0) / x2)),
            "rel_residual_compressed": float(np.sqrt(e_full / x2)), "rel_residual_direct": float(np.sqrt(e_dir / x2))}


def run_kernel(which):
    """A few launches of one kernel on the workload (for ncu captures): the
    first twelve mixed-path GN steps (pcg: one persistent CP-CG launch per step), the
    bf16x3 all-mode MTTKRP (mttkrp), or the residual-form gradient (resid:
    tensor-core reconstruction of E, then the MTTKRP of E)."""
    import torch

    from paper_1910_12331_gb300 import api, datagen

    p = datagen.workload(WORKLOAD, seed=0)
    dev = torch.device("cuda", 0)
    X = torch.from_numpy(p["X"]).to(dev)
    init = [torch.from_numpy(a.copy()).to(dev) for a in p["init"]]
    h = api.Handle(dev)
    if which == "mttkrp":
        M = [torch.empty_like(a) for a in init]
        for _ in range(3):
            api.cp_mttkrp_all(h, X, init, M, prec="bf16x3")
    elif which == "mttkrp500":
        g = torch.Generator(device=dev).manual_seed(500)
        X5 = torch.rand((500, 500, 500), generator=g, device=dev, dtype=torch.float32)
        A5 = [torch.rand((500, 500), generator=g, device=dev, dtype=torch.float64) for _ in range(3)]
        M5 = [torch.empty_like(a) for a in A5]
        for _ in range(2):
            api.cp_mttkrp_all(h, X5, A5, M5, prec="bf16x3")
    elif which == "resid":
        for _ in range(3):
            api.cp_gradient(h, X, init, prec="residual")
    else:
        lam_hi, lam_lo = lam_thresholds(p["init"])
        params = api.gn_params(lam_hi, lam_lo, lam_hi, MU, EPS_CG, CG_MAX, **MIXED)
        A = [a.clone() for a in init]
        for k in range(12):  # twelve GN steps of the solve: launches 11-12 run tens of CG iterations
            _, st = api.cp_gn_step(h, X, A, params, check=False)
            print("pcg launch %d: %d CG iterations" % (k + 1, st["cg_iters"]), flush=True)
    torch.cuda.synchronize()
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", choices=["pcg", "mttkrp", "mttkrp500", "resid"], default=None,
                    help="profiling aid: only run a few launches of one kernel on the workload, print nothing")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel:
        return run_kernel(args.kernel)

    import torch

    from paper_1910_12331_gb300 import api, datagen

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    p = datagen.workload(WORKLOAD, seed=0)
    X_host = torch.from_numpy(p["X"]).pin_memory()
    init_host = [torch.from_numpy(a.copy()).pin_memory() for a in p["init"]]
    X = X_host.to(dev)
    init = [a.to(dev) for a in init_host]
    A = [torch.empty_like(a) for a in init]
    lam_hi, lam_lo = lam_thresholds(p["init"])
    h = api.Handle(dev)
    total = int(np.prod(X.shape))
    R = init[0].shape[1]

    def solve(mode):
        for a, b in zip(A, init):
            a.copy_(b)
        h.bump_version(X)  # any cached split of X is rebuilt inside the timed step
        kw = MIXED if mode == "mixed" else {"prec": "fp64"}
        params = api.gn_params(lam_hi, lam_lo, lam_hi, MU, EPS_CG, CG_MAX, **kw)
        opts = api.solve_opts(max_iters=MAX_GN, target_stationarity=TARGET_STAT)
        _, res = api.cp_gn_solve(h, X, A, params, opts)
        return res

    def barrier():
        torch.cuda.synchronize()
        if pg:
            pg.barrier()

    # ---- warm-up and timed steps (mixed path); the clock sampler starts before the
    # warm-up so that nvidia-smi's start-up does not fall into the timed region
    with ClockSampler(local) as clk:
        clk.wait_first()
        for _ in range(args.warmup):
            solve("mixed")
        results = []
        barrier()
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        i0 = clk.mark()
        e0.record(stream)
        for _ in range(args.steps):
            results.append(solve("mixed"))
        e1.record(stream)
        barrier()
        i1 = clk.mark()
    t_total = e0.elapsed_time(e1) / 1e3
    t_step = t_total / args.steps
    t_step = max_over_ranks(t_step, pg, dev)
    last = results[-1]
    converged = all(r["converged"] for r in results)

    # ---- MTTKRP throughput (split planes resident; inputs larger than L2)
    M = [torch.empty_like(a) for a in init]
    api.cp_mttkrp_all(h, X, init, M, prec="bf16x3")
    n_mt = 20
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    m0.record(stream)
    for _ in range(n_mt):
        api.cp_mttkrp_all(h, X, init, M, prec="bf16x3")
    m1.record(stream)
    torch.cuda.synchronize()
    t_mt = m0.elapsed_time(m1) / 1e3 / n_mt
    mt_flops = 4.0 * total * R
    mt_bytes = 4.0 * total  # two bf16 planes of X read once
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    # ---- the plain FP64 path on the same problem (one solve)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    f0.record(stream)
    res64 = solve("fp64")
    f1.record(stream)
    torch.cuda.synchronize()
    t64 = f0.elapsed_time(f1) / 1e3

    # ---- end to end through the public API with host buffers
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    tw0 = time.perf_counter()
    for _ in range(e2e_steps):
        Xd = X_host.to(dev, non_blocking=True)
        Ad = [a.to(dev, non_blocking=True) for a in init_host]
        h.bump_version(Xd)
        params = api.gn_params(lam_hi, lam_lo, lam_hi, MU, EPS_CG, CG_MAX, **MIXED)
        opts = api.solve_opts(max_iters=MAX_GN, target_stationarity=TARGET_STAT)
        api.cp_gn_solve(h, Xd, Ad, params, opts)
        out = [a.cpu() for a in Ad]
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - tw0) / e2e_steps
    del Xd
    h2d = X_host.numel() * 4 + sum(a.numel() * 8 for a in init_host)
    d2h = sum(a.numel() * 8 for a in out)

    # ---- CP loss autograd Function (256^3 FP32, R=32): forward + fused-MTTKRP backward vs an einsum baseline
    loss_info = cp_loss_timing(dev)
    batch_info = batched_timing(dev)
    c3_info = c3_timing(dev)
    larger_info = large_r_mttkrp(dev)
    tucker_info = tucker_study(dev, A)
    exact_info = exact_cp_study(dev)

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return

    # roofline of the dominant phase inside the timed solve: the gradient of every GN iteration
    # (reconstruction of E on the tensor cores + the tensor-core MTTKRP of E), timed with CUDA events on
    # the handle's stream around the phase.  Algorithmic bytes of a gradient: one read of the FP32 X
    # (4 B per element); the planes of E written and read back are this design's own traffic, counted
    # in `traffic` (ncu DRAM bytes of the phase's kernels per gradient) and not in `achieved`.
    n_grad = last["iters"] + (1 if last["converged"] else 0)
    grad_s = last["mttkrp_ms"] / 1e3 / max(n_grad, 1)
    alg_bytes = 4.0 * total
    ach = alg_bytes / grad_s / 1e9
    rec = profiled("gradient")
    roof = {"kernel": "gradient phase of a GN iteration: recon_tc_kernel (E = X - [[A]]) + mttkrp_tc_kernel on E",
            "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": rec["dram_bytes"] if rec else None, "algorithmic_bytes": alg_bytes,
            "us_per_gradient": grad_s * 1e6, "gradients": n_grad, "peak_source": "measured (MEASURED_PEAKS.json)"}
    # the CG kernel: latency-bound; its floor is three grid barriers per iteration
    cg_it = max(last["cg_iters_total"], 1)
    pcg_s = last["pcg_ms"] / 1e3
    barrier_us = api.cp_probe_grid_barrier(local, last["cg_blocks"], 512)
    cg_roof = {"kernel": "pcg_kernel<float>", "bound": "latency (grid barriers)",
               "us_per_cg_iteration": pcg_s / cg_it * 1e6, "barrier_us": barrier_us, "blocks": last["cg_blocks"],
               "floor_us": 3 * barrier_us, "frac": 3 * barrier_us / (pcg_s / cg_it * 1e6),
               "cg_iterations": cg_it}
    # the plain FP64 path: FP64-ALU-bound; its MTTKRP against the measured DFMA rate
    fp64_peak = api.cp_probe_fp64_fma(local)
    Xf = X.double()
    api.cp_mttkrp_all(h, Xf, init, M, prec="fp64")
    torch.cuda.synchronize()
    m0.record(stream)
    for _ in range(5):
        api.cp_mttkrp_all(h, Xf, init, M, prec="fp64")
    m1.record(stream)
    torch.cuda.synchronize()
    t_mt64 = m0.elapsed_time(m1) / 1e3 / 5
    del Xf
    fp64_roof = {"kernel": "FP64 all-mode MTTKRP (mttkrp_y/z_kernel)", "bound": "fp64 alu",
                 "achieved": mt_flops / t_mt64 / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                 "frac": mt_flops / t_mt64 / 1e12 / fp64_peak, "us": t_mt64 * 1e6,
                 "peak_source": "measured (cp_probe_fp64_fma)"}
    cpu = None
    c1_info = c1_timing(dev)
    like_info = likelihood_study(dev)
    mm_info = matmul_study(dev)
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_record(p, lam_hi, lam_lo)
        c3_info["cpu_baseline"] = c3_cpu_sample()
        exact_info["cpu_baseline"] = exact_cp_cpu_sample()
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3/f32/f64", "data": "synthetic",
        "config": dict(CONFIG, parallelism=f"replicas x{ws}"),
        "converged": converged, "gn_iters": last["iters"], "gradient": "residual form -E_(n) P^(n) every iteration",
        "cg_iters": last["cg_iters_total"], "stationarity": last["stationarity"],
        "phase_ms": {"mttkrp": last["mttkrp_ms"], "pcg": last["pcg_ms"], "device": last["device_ms"]},
        "mttkrp": {"tflops": mt_flops / t_mt / 1e12, "us": t_mt * 1e6, "gbs": mt_bytes / t_mt / 1e9,
                   "hbm_frac": mt_bytes / t_mt / 1e9 / hbm_peak, "prec": "bf16x3"},
        "fp64_path": {"time_to_target_s": t64, "gn_iters": res64["iters"], "converged": bool(res64["converged"]),
                      "speedup_of_mixed": t64 / t_step},
        "roofline": roof,
        "roofline_cg": cg_roof,
        "roofline_fp64": fp64_roof,
        "cpu_baseline": cpu,
        "e2e": {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "cp_loss": loss_info,
        "batched": batch_info,
        "c1_exact20": c1_info,
        "c3_order4": c3_info,
        "mttkrp_large_rank": larger_info,
        "convergence_likelihood": like_info,
        "matmul_tensor": mm_info,
        "tucker_compressed": tucker_info,
        "exact_cp_rank_above_sides": exact_info,
        "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
        "clocks": clk.summary(i0, i1),
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
