#!/usr/bin/env python
"""Benchmark: time to solve A x = b to rtol 1e-8 on one GB300, plus BSR SpMV HBM GB/s.

Workload: the 256x256x128 channelised grid (8,388,608 cells, 25.2M unknowns,
4.2 GB of FP64 blocks; log-normal permeability with sigma 2, five x-aligned
streaks, 16 seeded wells, seed 2), solved by GMRES(30) + CPR-PF (quasi-IMPES,
geometric-multigrid V-cycle, block ILU(0)) to a true FP64 relative residual
of 1e-8.  One step = preconditioner setup + solve from x0 = 0 with the matrix
and right-hand side already resident in HBM, in the mixed-precision form
(FP32 inner solves under FP64 iterative refinement); the plain FP64 solve of
the same system is timed beside it over --fp64-steps solves.  The matrix is
far larger than the 129 MB L2, so no flush is needed between steps.
`--workload mid_100x100x50 --pc bilu0` runs the 100x100x50 layered workload
with block ILU(0) instead.

Prints one JSON line (rank 0).  `--impl reference` times the CPU FP64 oracle
(OpenMP build, every host core) instead, on bounded samples of the same
workload projected to the full solve.  Multi-GPU (torchrun): independent
replicas, one per GPU, timed together; the solver has no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve time to rtol 1e-8 + SpMV HBM GB/s; mixed/learned vs plain FP64 on 1 GB300"
WORKLOAD = "large_256x256x128"
PC = "cpr"
MID = "mid_100x100x50"
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129e6


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBps", "hbm"):
            if key in d and isinstance(d[key], (int, float)):
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def spmv_bytes(nb, nnzb, val_bytes=8):
    """Algorithmic bytes of one SpMV: blocks + column indices + row pointers + x + y."""
    return nnzb * (9 * val_bytes + 4) + (nb + 1) * 4 + 2 * nb * 3 * val_bytes


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture, with the
# kernel sources and their hash at capture time: a figure is reported only while the sources are unchanged.
# The ILU(0) apply's figure sums its three launches (gather, forward sweep, backward sweep).
NCU_TRAFFIC = {
    "ilu_apply_f32_large_256x256x128": (3429493000, ("ilu_tiles.cu", "common.cuh"), "f2ec801b4cf68fdb"),
    "spmv_f32_large_256x256x128": (2569320000, ("spmv.cu", "common.cuh"), "e5dfb24bef10827e"),
}


def spmv_flops(nnzb):
    return 2 * 9 * nnzb


def ilu_apply_bytes(nb, nnzb, val_bytes=8):
    """Algorithmic bytes of one block ILU(0) apply: every off-diagonal block once (lower
    blocks forward, upper backward), D^{-1} twice, r read, y written, y read, z written."""
    return (nnzb - nb) * 9 * val_bytes + 2 * nb * 9 * val_bytes + 4 * nb * 3 * val_bytes


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.dev = device_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(device_index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def max_over_ranks(ms, dist, dev=None):
    """The slowest rank's time (every rank gets it), then a barrier; ms itself when single-process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def golden_iters(workload, key):
    """The oracle's own iteration count on a workload (tests/golden/oracle_solves.json, written by
    tests/golden/make_golden.py from the oracle alone), or None."""
    gold = os.path.join(ROOT, "tests", "golden", "oracle_solves.json")
    try:
        return int(json.load(open(gold))[f"{workload}/{key}"]["iters"])
    except (OSError, KeyError, ValueError):
        return None


class OracleSample:
    """The oracle (as it stands, its OpenMP build at every host core) on a bounded sample of the
    workload: one preconditioner setup, then GMRES(30) runs of `sample_iters` iterations from
    x0 = 0.  The full solve's time is projected as setup + per-iteration time x the oracle's own
    full iteration count.  The sample's iterations are the first of a restart cycle, whose
    Gram-Schmidt work is below a cycle's average; the preconditioner dominates each iteration."""

    def __init__(self, p, pc, full_iters, threads=None, coarsening="gmg"):
        import oracle
        self.threads = oracle.use_threads(threads or os.cpu_count() or 1)
        self.p, self.full_iters = p, full_iters
        t0 = time.perf_counter()
        kw = {"coarsening": "amg", "gmg_levels": 8} if coarsening == "amg" else {}
        self.sys = oracle.System.from_problem(p, pc=pc, **kw)
        self.setup_s = time.perf_counter() - t0

    def run(self, sample_iters):
        t0 = time.perf_counter()
        _, _, info = self.sys.gmres(self.p.b, m=30, maxit=sample_iters)
        dt = time.perf_counter() - t0
        return dt, max(info["iters"], 1)

    def projected_ms(self, per_iter_s):
        return 1e3 * (self.setup_s + per_iter_s * self.full_iters)


def cpu_baseline(p, workload, pc, full_iters, sample_iters, coarsening="gmg"):
    """cpu_baseline entry of the bench line: one OracleSample run."""
    t_all = time.perf_counter()
    o = OracleSample(p, pc, full_iters, coarsening=coarsening)
    dt, done = o.run(sample_iters)
    per_iter = dt / done
    return {"value": round(o.projected_ms(per_iter), 3), "unit": "ms", "cores": o.threads, "kind": "oracle",
            "cpu": cpu_model(), "build": "oracle.c with OpenMP (SpMV rows, vector updates, one colour of "
            "Gauss-Seidel, stencil products in parallel; ILU(0) sweeps sequential)",
            "sample": f"oracle setup ({o.setup_s:.1f} s) + the first {done} GMRES(30)+{pc.upper()} iterations "
                      f"on {workload} at {o.threads} threads ({per_iter:.2f} s each; "
                      f"{time.perf_counter() - t_all:.1f} s of CPU work), projected to the oracle's "
                      f"{full_iters} iterations of the full FP64 solve"}


def run_reference(args, rank, ws):
    """The reference arm: the CPU oracle on the same workload and config as the GPU arm.  Each
    timed step is a bounded sample (args.ref_sample_iters GMRES iterations); the line's value
    projects the per-iteration time of all timed steps to the oracle's full solve."""
    if rank != 0:
        return 0
    import synth
    p = synth.workload(args.workload)
    full_iters = golden_iters(args.workload, f"gmres/{pc_key(args)}")
    if full_iters is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no recorded oracle iteration count for "
                          f"{args.workload} gmres/{pc_key(args)}"}), flush=True)
        return 0
    o = OracleSample(p, args.pc, full_iters, coarsening=args.coarsening)
    for _ in range(args.warmup):
        o.run(max(1, args.ref_sample_iters // 2))
    t0 = time.perf_counter()
    tot_s, tot_it = 0.0, 0
    for _ in range(args.steps):
        dt, done = o.run(args.ref_sample_iters)
        tot_s += dt
        tot_it += done
    wall_s = time.perf_counter() - t0
    per_iter = tot_s / max(tot_it, 1)
    v = round(o.projected_ms(per_iter), 3)
    step_ms = round(1e3 * wall_s / max(args.steps, 1), 3)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(p, args.workload, pc_key(args), ws),
            "value_is_projection": True,
            "projection": f"value = oracle setup ({o.setup_s:.1f} s) + mean time per GMRES iteration over the "
                          f"{args.steps} timed steps ({per_iter:.3f} s) x the oracle's {full_iters} iterations of "
                          f"the full FP64 solve; ms_per_step is the measured time of one sampled step",
            "cpu_baseline": {"value": v, "unit": "ms", "cores": o.threads, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"each step: the first {args.ref_sample_iters} GMRES(30)+"
                                       f"{args.pc.upper()} iterations from x0 = 0 (FP64 oracle, OpenMP build)"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """The batched-ensemble workload: 64 independent systems solved by one batched call."""
    import numpy as np
    import torch

    import paper_1602_05901_gb300 as rsv
    import synth
    dims = synth.batch_sizes()
    t0 = time.perf_counter()
    probs = [synth.make_problem(*d, seed=1000 + q) for q, d in enumerate(dims)]
    vals = np.concatenate([p.vals for p in probs])
    b = np.concatenate([p.b for p in probs])
    gen_s = time.perf_counter() - t0
    A = rsv.Matrix.batch(dims)
    A.set_values(torch.from_numpy(vals).cuda())
    s = rsv.Solver(A, solver="bicgstab", precision="mixed", rtol=1e-8, maxit=4000)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)

    def step():
        s.setup("bilu0")
        x.zero_()
        st, infos = s.solve_batched(bd, x)
        if st != rsv.RSV_OK:
            raise RuntimeError(f"batched solve: {rsv.status_string(st)}")
        return infos

    for _ in range(max(args.warmup, 1)):
        infos = step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = rsv.rsv_kernel_launches()
    e0.record()
    for _ in range(args.steps):
        infos = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    its = [i["iters"] for i in infos]
    rel = [i["true_relres"] for i in infos]
    line = {"workload": "batch64_uneven", "metric": "batched solve time to rtol 1e-8 (all 64 systems)",
            "value": round(ms, 3), "unit": "ms", "higher_is_better": False, "steps": args.steps,
            "systems": len(dims), "cells": int(A.nb), "unknowns": int(3 * A.nb),
            "systems_per_s": round(len(dims) / (ms * 1e-3), 1),
            "iters_min_median_max": [int(min(its)), int(np.median(its)), int(max(its))],
            "max_true_relres": float(max(rel)), "gpu_launches_per_step": int((rsv.rsv_kernel_launches() - l0) / args.steps),
            "generation_s": round(gen_s, 1),
            "config": {"solver": "bicgstab", "pc": "bilu0 (batched tile sweeps)",
                       "precision": "FP32 inner + FP64 refinement", "graph": "CUDA graph of 4 passes"}}
    print(json.dumps(line), flush=True)
    return 0


def unet_flops(nx, ny, nz, base=32, levels=4):
    """(forward flops, training-step flops) of the U-Net, counted from its layers.

    A 3x3x3 layer costs 2*V*co*ci*27 per pass; the first layer's 27 taps x 2 input
    channels count as K = 54 (its padding to 64 is not counted).  Training runs the
    forward pass, the input gradient of every layer but the first, and every
    weight gradient.
    """
    ch = [base << l for l in range(levels)]
    V = [(nx >> l) * (ny >> l) * (nz >> l) for l in range(levels)]
    layers = []  # (V, co, K)
    prev = 2
    for l in range(levels):
        layers += [(V[l], ch[l], prev * 27), (V[l], ch[l], ch[l] * 27)]
        prev = ch[l]
    for l in range(levels - 2, -1, -1):
        layers += [(V[l], ch[l], (ch[l + 1] + ch[l]) * 27), (V[l], ch[l], ch[l] * 27)]
    fwd = sum(2.0 * v * co * k for v, co, k in layers) + 2.0 * V[0] * ch[0]
    dgrad = sum(2.0 * v * co * k for v, co, k in layers[1:])
    return fwd, fwd + dgrad + fwd


def tc_peak():
    """Dense BF16 tensor peak (TFLOP/s): MEASURED_PEAKS.json when present, else the recipe's fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def run_unet(args):
    """Time the learned stage's network at 128x128x64: one application and one training step."""
    import numpy as np
    import torch

    import paper_1602_05901_gb300 as rsv
    import synth
    nx, ny, nz = 128, 128, 64
    net = rsv.Unet(nx, ny, nz, base=32, levels=4)
    net.set_params(synth.unet_init(32, 4, seed=0))
    g = torch.Generator(device="cuda").manual_seed(0)
    V = nx * ny * nz
    rp = torch.randn(V, dtype=torch.float64, device="cuda", generator=g)
    lnk = torch.randn(V, dtype=torch.float64, device="cuda", generator=g)
    tgt = torch.randn(V, dtype=torch.float64, device="cuda", generator=g) * 0.05
    out = torch.empty_like(rp)
    fwd_f, train_f = unet_flops(nx, ny, nz)

    def timed(fn, k):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    ms_apply = timed(lambda: net.apply(rp, lnk, out), args.steps)
    ms_train = timed(lambda: net.train_batch([rp] * 8, [lnk] * 8, [tgt] * 8, 1e-4), args.steps) / 8
    peak, src = tc_peak()
    line = {"workload": "unet_128x128x64_base32_L4", "metric": "U-Net application and training step",
            "apply_ms": round(ms_apply, 3), "apply_tflops": round(fwd_f / ms_apply * 1e-9, 1),
            "train_step_ms": round(ms_train, 3), "train_tflops": round(train_f / ms_train * 1e-9, 1),
            "flops_apply": fwd_f, "flops_train_step": train_f, "peak_bf16_tflops": peak, "peak_source": src,
            "apply_frac_of_peak": round(fwd_f / ms_apply * 1e-9 / peak, 4),
            "params": int(net.nparam), "dtype": "bf16 operands, fp32 accumulate"}
    print(json.dumps(line), flush=True)
    return 0


def run_cpr_orders(args):
    """The four CPR stage orders (PF, FP, FPF, FFPF) with quasi-IMPES and ABF decoupling as
    GMRES(30) preconditioners on the benchmark workload, FP64 and mixed precision: setup +
    solve to rtol 1e-8, CUDA events on the solver stream, `--warmup` untimed and `--steps`
    timed solves per combination."""
    import torch

    import paper_1602_05901_gb300 as rsv
    import synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p = synth.workload(MID)
    stream = torch.cuda.current_stream(dev).cuda_stream
    A = rsv.Matrix(p.nx, p.ny, p.nz, stream=stream)
    A.set_values(torch.from_numpy(p.vals).to(dev))
    b = torch.from_numpy(p.b).to(dev)
    x = torch.zeros_like(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    combos = [(d, pr, pc) for d in ("qi", "abf") for pr in ("fp64", "mixed")
              for pc in ("cpr", "cpr_fp", "cpr_fpf", "cpr_ffpf")]
    for decoupling, precision, pc in combos:
        s = rsv.Solver(A, solver="gmres", restart=30, rtol=1e-8, maxit=4000, precision=precision)

        def step():
            s.setup(pc, decoupling=decoupling)
            x.zero_()
            st, info = s.solve(b, x)
            if st != rsv.RSV_OK:
                raise RuntimeError(f"{pc} {precision}: {rsv.status_string(st)} {info}")
            return info
        for _ in range(max(1, args.warmup)):
            step()
        torch.cuda.synchronize(dev)
        e0.record()
        infos = [step() for _ in range(args.steps)]
        e1.record()
        torch.cuda.synchronize(dev)
        rows.append({"pc": pc, "decoupling": decoupling, "precision": precision,
                     "ms": round(e0.elapsed_time(e1) / args.steps, 3),
                     "iters": infos[-1]["iters"], "outer_iters": infos[-1].get("outer_iters", 0),
                     "true_relres": infos[-1]["true_relres"]})
    print(json.dumps({"mode": "cpr-orders", "workload": MID, "solver": "gmres(30)", "rtol": 1e-8,
                      "steps": args.steps, "warmup": args.warmup, "results": rows}))
    return 0


def run_learned(args):
    """The learned pressure stage on the 128x128x64 channelised workload.

    Training: the pressure-stage inputs of plain FP64 FGMRES(30) + CPR solves of
    ``--learned-train`` seeded systems (the first 40 CPR applications of each),
    V-cycle targets, ``--learned-epochs`` epochs of Adam.  Evaluation on
    ``--learned-eval`` unseen seeds: FP64 GMRES(30) + CPR (the V-cycle) against
    FP64 FGMRES(30) + learned CPR (with its fallback) and FGMRES(30) + block ILU(0)
    (the method without a pressure stage), each to rtol 1e-8; time = setup + solve.
    """
    import numpy as np
    import torch

    import paper_1602_05901_gb300 as rsv
    import synth
    from paper_1602_05901_gb300 import learned as Lr
    grid = (128, 128, 64)
    t0 = time.perf_counter()
    samples, gen_s = [], 0.0
    for q in range(args.learned_train):
        tg = time.perf_counter()
        p = synth.workload("learned_128x128x64", seed=20000 + q)
        gen_s += time.perf_counter() - tg
        rp, tgt = Lr.collect_samples(grid, p.vals, p.b, 40)
        lnk = torch.tensor(p.lnk, device="cuda")
        samples += [(rp[i], lnk, tgt[i]) for i in range(rp.shape[0])]
        del p
    collect_s = time.perf_counter() - t0 - gen_s
    net = rsv.Unet(*grid, base=32, levels=4)
    net.set_params(synth.unet_init(32, 4, seed=0))
    _, train_f = unet_flops(*grid)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    losses = Lr.train(net, samples, args.learned_epochs, lr=3e-4, seed=0)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    steps = len(samples) * args.learned_epochs
    rows = []
    imit = None
    for q in range(args.learned_eval):
        p = synth.workload("learned_128x128x64", seed=30000 + q)
        if q == 0:
            rpe, tge = Lr.collect_samples(grid, p.vals, p.b, 20)
            imit = float(Lr.imitation_error(net, rpe, torch.tensor(p.lnk, device="cuda"), tge).mean())
            del rpe, tge
        A = rsv.Matrix(*grid)
        A.set_values(p.vals)
        for solver, pc in (("gmres", "cpr"), ("fgmres", "cpr_learned"), ("fgmres", "bilu0")):
            s = rsv.Solver(A, solver=solver, precision="fp64", rtol=1e-8, maxit=4000)
            if pc == "cpr_learned":
                # stall window of one restart cycle: plain CPR itself falls only ~2% per iteration
                # on this workload, so the 10%-over-5 default would flag any preconditioner
                s.set_learned(net, p.lnk, stall_window=30, stall_drop=0.10)
            s.setup(pc)
            x = np.zeros(3 * p.nb)
            st, info = s.solve(p.b.copy(), x)
            rows.append({"seed": 30000 + q, "solver": solver, "pc": pc, "status": st, "iters": info["iters"],
                         "ms": round(info["ms_setup"] + info["ms_solve"], 1),
                         "true_relres": info["true_relres"], "fallback_iter": info["fallback_iter"]})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            del s
        del A, p

    def med(pc, key):
        v = [r[key] for r in rows if r["pc"] == pc and r["status"] == 0]
        return float(statistics.median(v)) if v else None

    line = {"workload": "learned_128x128x64 (channelised sigma 2, 16 seeded wells)",
            "metric": "time to rtol 1e-8 (FP64 true residual), median over unseen seeds", "unit": "ms",
            "higher_is_better": False,
            "plain_cpr_gmres_ms": med("cpr", "ms"), "learned_cpr_fgmres_ms": med("cpr_learned", "ms"),
            "bilu0_fgmres_ms": med("bilu0", "ms"),
            "plain_cpr_iters": med("cpr", "iters"), "learned_cpr_iters": med("cpr_learned", "iters"),
            "bilu0_iters": med("bilu0", "iters"),
            "learned_fallbacks": sum(1 for r in rows if r["pc"] == "cpr_learned" and r["fallback_iter"] >= 0),
            "all_converged": all(r["status"] == 0 and r["true_relres"] <= 1e-8 for r in rows),
            "stall_rule": "fall back when the implicit residual falls < 10% over 30 iterations",
            "eval_seeds": args.learned_eval, "train_systems": args.learned_train, "train_samples": len(samples),
            "epochs": args.learned_epochs, "loss_first_last_epoch": [losses[0], losses[-1]],
            "imitation_error_unseen": imit,
            "train_step_ms": round(train_ms / steps, 3), "train_tflops": round(train_f * steps / train_ms * 1e-9, 1),
            "generation_s": round(gen_s, 1), "sample_collection_s": round(collect_s, 1), "runs": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_conv():
    """One launch of each hot convolution on the network's finest level (128x128x64, 32 and 96 channels),
    for ncu captures; checks that the outputs are finite.  Prints no benchmark line."""
    import ctypes

    import torch

    import paper_1602_05901_gb300 as rsv
    nx, ny, nz = 128, 128, 64
    V = nx * ny * nz
    g = torch.Generator(device="cuda").manual_seed(0)
    x = (torch.randn(V, 96, device="cuda", generator=g)).to(torch.bfloat16)
    w = (torch.randn(32, 27, 96, device="cuda", generator=g) * 0.02).to(torch.bfloat16)
    y = torch.empty(V, 32, dtype=torch.bfloat16, device="cuda")
    gw = torch.empty(32, 27, 96, device="cuda")
    gb = torch.empty(32, device="cuda")
    gx = torch.empty(V, 96, dtype=torch.bfloat16, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rsv.check(rsv.rsv_conv3d_fwd(None, nx, ny, nz, 27, 32, 32, p(x), 96, p(w), None, 1, None, 0, p(y), 32, None))
    rsv.check(rsv.rsv_conv3d_fwd(None, nx, ny, nz, 27, 96, 32, p(x), 96, p(w), None, 1, None, 0, p(y), 32, None))
    rsv.check(rsv.rsv_conv3d_dgrad(None, nx, ny, nz, 96, 32, p(y), 32, p(w), None, 0, p(gx), 96, None))
    rsv.check(rsv.rsv_conv3d_wgrad(None, nx, ny, nz, 27, 96, 32, p(x), 96, p(y), 32, p(gw), p(gb)))
    torch.cuda.synchronize()
    assert torch.isfinite(y.float()).all() and torch.isfinite(gx.float()).all() and torch.isfinite(gw).all()
    print("profile-conv done", flush=True)
    return 0


def run_profile_mode(args):
    """Small, self-checking runs of the hot path for ncu (no timing is reported)."""
    import torch

    import paper_1602_05901_gb300 as rsv
    import synth
    mode = args.mode
    p = synth.workload(args.workload)
    A = rsv.Matrix(p.nx, p.ny, p.nz)
    A.set_values(p.vals)
    if mode == "profile-solve":
        s = rsv.Solver(A, solver="gmres", restart=30, rtol=1e-8, maxit=60, precision="mixed")
        s.setup(args.pc, **pc_kwargs(args))
        b = torch.from_numpy(p.b).cuda()
        x = torch.zeros_like(b)
        st, info = s.solve(b, x)
        torch.cuda.synchronize()
        assert st in (rsv.RSV_OK, rsv.RSV_ENOCONV), st
        print("profile-solve", info)
        return 0
    s32 = rsv.Solver(A, precision="mixed")
    s32.setup("bilu0")
    s64 = rsv.Solver(A, precision="fp64")
    s64.setup("bilu0")
    x = torch.randn(p.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    x32, y32 = x.float(), torch.empty(p.n, dtype=torch.float32, device="cuda")
    for _ in range(3):
        A.spmv(x, y)
        A.spmv(x32, y32)
        s32.apply(x32, y32)
        s64.apply(x, y)
    torch.cuda.synchronize()
    print("profile-kernels done")
    return 0


PC_DESC = {"cpr": "CPR-PF: quasi-IMPES, GMG V-cycle (2 red-black sweeps, <= 6 levels), block ILU(0) "
                  "(i+j+k wavefront tiles)",
           "cpr-amg": "CPR-PF: quasi-IMPES, AMG V-cycle (PMIS, direct interpolation, 2 l1-Jacobi sweeps, <= 8 "
                      "levels), block ILU(0) (i+j+k wavefront tiles)",
           "bilu0": "block ILU(0) (i+j+k wavefront tiles)"}


def pc_kwargs(args):
    """Preconditioner parameters of the run: the pressure stage's coarsening for CPR."""
    if args.pc == "cpr" and args.coarsening == "amg":
        return {"coarsening": "amg", "gmg_max_levels": 8}
    return {}


def pc_key(args):
    return "cpr-amg" if args.pc == "cpr" and args.coarsening == "amg" else args.pc
MOBILITY_READING = ("M_ij: off-diagonal entries U(0.1,1), each diagonal entry U(0.1,1) plus its row's three draws "
                    "(row-diagonally dominant); nine i.i.d. U(0.1,1) entries make the Jacobian indefinite")


def bench_config(p, workload, pc, ws):
    return {"workload": workload, "grid": [p.nx, p.ny, p.nz], "cells": p.nb, "unknowns": p.n, "nnzb": p.nnzb,
            "solver": "gmres(30)", "pc": PC_DESC[pc], "rtol": 1e-8, "x0": "zero",
            "precision": "value: FP32 inner solves (inner rtol 1e-5; the last step only to what the target "
                         "needs) under FP64 refinement; fp64: plain FP64",
            "mobility_reading": MOBILITY_READING, "parallelism": f"replicas x{ws}",
            "l2": f"inputs larger than L2 (FP64 blocks {p.vals.nbytes / 1e6:.0f} MB > 129 MB), no flush"}


def source_sha(*names):
    """Short hash of kernel sources: a recorded ncu traffic figure holds only for the sources it was taken on."""
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1602_05901_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(key):
    """DRAM bytes per launch from one ncu capture (read + write), or None when the kernel's sources
    changed since the capture."""
    entry = NCU_TRAFFIC.get(key)
    if not entry:
        return None
    traffic, srcs, sha = entry
    return traffic if source_sha(*srcs) == sha else None


def run_bench(args, rank, ws, local, dist):
    import numpy as np  # noqa: F401
    import torch

    import paper_1602_05901_gb300 as rsv
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p = synth.workload(args.workload)
    A = rsv.Matrix(p.nx, p.ny, p.nz, stream=stream)
    vals_d = torch.from_numpy(p.vals).to(dev)
    A.set_values(vals_d)
    del vals_d
    b = torch.from_numpy(p.b).to(dev)
    x = torch.zeros_like(b)
    s = rsv.Solver(A, solver="gmres", restart=30, rtol=1e-8, maxit=6000, precision="mixed")
    s64 = rsv.Solver(A, solver="gmres", restart=30, rtol=1e-8, maxit=6000, precision="fp64")

    def step(solver):
        solver.setup(args.pc, **pc_kwargs(args))
        x.zero_()
        st, info = solver.solve(b, x)
        if st != rsv.RSV_OK:
            raise RuntimeError(f"solve failed: {rsv.status_string(st)} {info}")
        return info

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(solver, steps):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        l0 = rsv.rsv_kernel_launches()
        e0.record(stream)
        infos = [step(solver) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_ = max_over_ranks(e0.elapsed_time(e1) / steps, dist, dev)
        return ms_, infos[-1], rsv.rsv_kernel_launches() - l0

    fp64_steps = max(1, min(args.steps, args.fp64_steps))
    for _ in range(args.warmup):
        step(s)
    step(s64)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    ms, info, launches = timed(s, args.steps)
    ms64, info64, _ = timed(s64, fp64_steps)
    clocks = sampler.stop()

    # ---- kernel microbenchmarks on the same stream (CUDA events)
    peak, peak_src = hbm_peak()

    def event_ms(fn, reps):
        for _ in range(3):
            fn()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    xs = torch.randn(p.n, dtype=torch.float64, device=dev)
    ys = torch.empty_like(xs)
    xs32, ys32 = xs.float(), torch.empty(p.n, dtype=torch.float32, device=dev)
    spmv_ms = event_ms(lambda: A.spmv(xs, ys), 30)
    spmv32_ms = event_ms(lambda: A.spmv(xs32, ys32), 30)
    sb, sb32 = spmv_bytes(p.nb, p.nnzb), spmv_bytes(p.nb, p.nnzb, 4)
    spmv_gbs, spmv32_gbs = sb / (spmv_ms * 1e-3) / 1e9, sb32 / (spmv32_ms * 1e-3) / 1e9
    # the mixed path's preconditioner stages, FP32: block ILU(0) alone and the whole CPR apply
    s_ilu = rsv.Solver(A, precision="mixed")
    s_ilu.setup("bilu0")
    zs32 = torch.empty_like(xs32)
    ilu32_ms = event_ms(lambda: s_ilu.apply(xs32, zs32), 10)
    del s_ilu
    s.setup(args.pc, **pc_kwargs(args))
    pc32_ms = event_ms(lambda: s.apply(xs32, zs32), 10)
    ib32 = ilu_apply_bytes(p.nb, p.nnzb, 4)
    ilu32_gbs = ib32 / (ilu32_ms * 1e-3) / 1e9
    # dominant kernel of the timed (mixed) path per inner iteration: the FP32 ILU(0) sweeps (one per
    # preconditioner application) against the FP32 SpMV (one per iteration, two with CPR)
    spmv_per_iter = 2 if args.pc == "cpr" else 1
    if ilu32_ms >= spmv_per_iter * spmv32_ms:
        dom = {"kernel": "block ILU(0) apply, FP32 (forward + backward tile sweeps)", "ms": ilu32_ms, "bytes": ib32,
               "gbs": ilu32_gbs, "traffic": recorded_traffic("ilu_apply_f32_" + args.workload)}
    else:
        dom = {"kernel": "BSR SpMV FP32", "ms": spmv32_ms, "bytes": sb32, "gbs": spmv32_gbs,
               "traffic": recorded_traffic("spmv_f32_" + args.workload)}
    roofline = {"bound": "hbm", "achieved": round(dom["gbs"], 1), "peak": peak, "unit": "GB/s",
                "frac": round(dom["gbs"] / peak, 4), "traffic": dom["traffic"], "kernel": dom["kernel"],
                "algorithmic_bytes_per_launch": dom["bytes"], "avg_launch_ms": round(dom["ms"], 4),
                "peak_source": peak_src}
    del xs, ys, xs32, ys32, zs32

    # ---- end to end through the C ABI with host buffers: values, b and x in, x out, every step
    vals_h = torch.from_numpy(p.vals).pin_memory()
    b_h = torch.from_numpy(p.b).pin_memory()
    x_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()

    def e2e_step():
        A.set_values(vals_h.numpy())
        s.setup(args.pc, **pc_kwargs(args))
        x_h.zero_()
        st, einfo = s.solve(b_h.numpy(), x_h.numpy())
        assert st == rsv.RSV_OK, rsv.status_string(st)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
    wall_e2e_ms = (time.perf_counter() - t0) * 1e3 / args.e2e_steps
    h2d = p.vals.nbytes + p.b.nbytes + p.b.nbytes
    d2h = p.b.nbytes
    del vals_h

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        full = golden_iters(args.workload, f"gmres/{pc_key(args)}") or info64["iters"]
        cpu = cpu_baseline(p, args.workload, args.pc, full, args.cpu_sample_iters, args.coarsening)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 inner / f64 refinement", "data": "synthetic",
            "config": bench_config(p, args.workload, pc_key(args), ws),
            "iters": info["iters"], "outer_iters": info["outer_iters"], "true_relres": info["true_relres"],
            "ms_setup": round(info["ms_setup"], 3), "ms_solve": round(info["ms_solve"], 3),
            "fp64": {"ms_per_step": round(ms64, 3), "steps": fp64_steps, "warmup": 1, "iters": info64["iters"],
                     "true_relres": info64["true_relres"], "ms_setup": round(info64["ms_setup"], 3),
                     "speedup_mixed_over_fp64": round(ms64 / ms, 3),
                     "oracle_iters": golden_iters(args.workload, f"gmres/{pc_key(args)}")},
            "oracle_refinement_iters": golden_iters(args.workload, f"refine-gmres/{pc_key(args)}"),
            "kernels": {"spmv_f64_ms": round(spmv_ms, 4), "spmv_f64_gbs": round(spmv_gbs, 1),
                        "spmv_f64_frac": round(spmv_gbs / peak, 4),
                        "spmv_f64_gflops": round(spmv_flops(p.nnzb) / (spmv_ms * 1e-3) / 1e9, 1),
                        "spmv_f32_ms": round(spmv32_ms, 4), "spmv_f32_gbs": round(spmv32_gbs, 1),
                        "spmv_f32_frac": round(spmv32_gbs / peak, 4), "spmv_algorithmic_bytes": [sb, sb32],
                        "ilu_apply_f32_ms": round(ilu32_ms, 4), "ilu_apply_f32_gbs": round(ilu32_gbs, 1),
                        "pc_apply_f32_ms": round(pc32_ms, 4)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "steps": args.e2e_steps,
                    "wall_ms": round(wall_e2e_ms, 3), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "path": "rsv_mat_set_values + rsv_precond_setup + rsv_solve_ptr on pinned host buffers"},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rsv", choices=["rsv", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=["large_256x256x128", "mid_100x100x50"])
    ap.add_argument("--pc", default=PC, choices=["cpr", "bilu0"])
    ap.add_argument("--coarsening", default="gmg", choices=["gmg", "amg"],
                    help="CPR's pressure hierarchy: geometric (default) or algebraic")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 solves (at most --steps)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-iters", type=int, default=10)
    ap.add_argument("--ref-sample-iters", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned-train", type=int, default=12, help="learned mode: training systems")
    ap.add_argument("--learned-epochs", type=int, default=20, help="learned mode: epochs")
    ap.add_argument("--learned-eval", type=int, default=4, help="learned mode: unseen evaluation seeds")
    ap.add_argument("--mode", default="bench",
                    choices=["bench", "profile-solve", "profile-kernels", "profile-conv", "batch", "unet", "learned",
                             "cpr-orders"],
                    help="profile-solve: one short mixed GMRES(30)+BILU0 solve (60 inner iterations) on the "
                         "benchmark workload, for an ncu launch list; profile-kernels: set up the benchmark "
                         "workload and run each hot kernel (FP64/FP32 SpMV, FP32/FP64 ILU(0) apply) three times, "
                         "for ncu captures. Neither prints a benchmark line. batch: time the 64-system "
                         "uneven ensemble (grids from 16^3 to 96x96x48, BiCGSTAB + block ILU(0), FP32 inner "
                         "solves under FP64 refinement, rtol 1e-8 per system) and print its own JSON line.")
    args = ap.parse_args()
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "unet":
        return run_unet(args)
    if args.mode == "profile-conv":
        return run_profile_conv()
    if args.mode == "cpr-orders":
        return run_cpr_orders(args)
    if args.mode == "learned":
        return run_learned(args)
    if args.mode != "bench":
        return run_profile_mode(args)
    if args.warmup < 3 and args.impl == "rsv":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    rank, ws, local, dist = dist_init()
    if args.impl == "reference":
        rc = run_reference(args, rank, ws)
        if dist is not None:
            dist.destroy_process_group()
        return rc
    rc = run_bench(args, rank, ws, local, dist)
    if dist is not None:
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
