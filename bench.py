#!/usr/bin/env python3
"""Benchmark of the Bi-cADMM hot path on one B300 (replicas on N GPUs).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Workload: sparse logistic regression, A 200000 x 5000 FP32 with Toeplitz column
correlation 0.3^|i-j|, 50-sparse planted model, labels sign(A x* + N(0, 0.5^2)),
N = 16 sample shards, M = 8 feature blocks, kappa = 50, rho = 0.5 (synthetic, seeded).
A step is one outer Bi-cADMM iteration (one inner sweep: x-update, fused A pass,
global (z,t,s,v) step, dual update).  `value` is outer iterations per second with A
resident in HBM; `e2e` is the same metric through the public C ABI from pinned host
buffers (create + setup + K iterations + get_x, H2D of A and b inside the timed region).

The default line also carries `legs.softmax` (the 500000 x 2000 x 10 BF16 softmax workload's
value, tensor-core pass roofline and end-to-end figure) and `legs.path` (10 logistic
instances at kappa 20..800 on one 500000 x 2000 BF16 A, one tensor-core pass per sweep for
all of them, against one single-kappa handle) and `legs.batch` (256 uneven FP32 instances
advanced by batched launches); skip them with --no-legs.

--impl reference times the FP64 CPU oracle on a bounded sample (one of the 16 shards): its
steps are shard iterations (steps x ms_per_step = the time spent) and its value is the
whole workload's rate extrapolated from them (`extrapolated`, `extrapolation_factor`).
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

from paper_2405_16267_b300 import synth  # noqa: E402

WORKLOAD = dict(name="sparse_logistic_200000x5000_fp32", m=200000, n=5000, nnz=50, corr=0.3,
                noise=0.5, N=16, M=8, kappa=50, rho=0.5, gamma=10.0, seed=0)
METRIC = "ADMM iters/s"
UNIT = "iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--m", type=int, default=None, help="override rows (profiling small cases)")
    ap.add_argument("--pass-rows", type=int, default=0)
    ap.add_argument("--pass-stages", type=int, default=0)
    ap.add_argument("--inner", type=int, default=1, help="inner sharing sweeps J per iteration")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance leg")
    ap.add_argument("--no-legs", action="store_true",
                    help="default workload only: skip the softmax, path and batch legs added to its line")
    ap.add_argument("--workload", default="logistic", choices=["logistic", "softmax", "batch", "serve", "path"],
                    help="softmax: 500000 x 2000 BF16, 10 classes (tensor-core pass); "
                         "batch: 256 uneven instances advanced by batched launches; "
                         "serve: a Poisson stream of solves through the serving loop")
    ap.add_argument("--requests", type=int, default=64, help="requests in the serve workload")
    ap.add_argument("--rate", type=float, default=200.0, help="mean arrivals/s (serve)")
    ap.add_argument("--serve-iters", type=int, default=100, help="iteration cap per request")
    ap.add_argument("--batch", type=int, default=256, help="instances in the batch workload")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="storage precision of A in the batch and serve workloads")
    return ap.parse_args()


def config_dict(wl, extra=None):
    d = {"workload": wl["name"], "m": wl["m"], "n": wl["n"], "N_shards": wl["N"],
         "M_blocks": wl["M"], "kappa": wl["kappa"], "rho": wl["rho"], "gamma": wl["gamma"],
         "loss": "logistic", "inner_iters": 1, "A_dtype": "f32",
         "l2": "inputs larger than L2 (A is %.1f GB)" % (wl["m"] * wl["n"] * 4 / 1e9),
         "parallelism": "replicas"}
    if extra:
        d.update(extra)
    return d


# ----------------------------------------------------------------------------- data

def generate(wl, rows=None):
    """Seeded FP32 A (pinned host tensor when torch is available) and labels b."""
    m = wl["m"]
    r0, r1 = (0, m) if rows is None else rows
    shards = synth.split_ranges(m, wl["N"])
    # generate shard by shard in a thread pool (the RNG and IIR filter release the GIL)
    from concurrent.futures import ThreadPoolExecutor
    pieces = []
    for (a, b_) in shards:
        lo, hi = max(a, r0), min(b_, r1)
        if lo < hi:
            pieces.append((lo, hi))
    out_A = np.empty((r1 - r0, wl["n"]), dtype=np.float32)
    out_b = np.empty(r1 - r0)

    def job(rng):
        lo, hi = rng
        P = synth.sparse_logistic(m=m, n=wl["n"], nnz=wl["nnz"], corr=wl["corr"],
                                  noise=wl["noise"], seed=wl["seed"], rows=(lo, hi))
        out_A[lo - r0:hi - r0] = P.A
        out_b[lo - r0:hi - r0] = P.b
        return P.x_star

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        xs = list(ex.map(job, pieces))
    return out_A, out_b, xs[0]


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, interval_ms=50):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        self.marks = []

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers

# DRAM traffic of one pass launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of a 20000-row launch of the same kernel, scaled by rows to the
# 200000-row launch.  Reported only while the kernel sources are the captured ones.
PASS_TRAFFIC = {"sources_sha256": "55c0b0a1e2e140e183d15c83d9823000ed48dfcc2b6d8bf539f9755eae87ffce", "bytes_per_launch": 4.0515e+09,
                "capture": "profiles/k_fused_pass_sparse_logistic_200000x5000_fp32.md"}
PASS_SOURCES = ["paper_2405_16267_b300/csrc/pass.cuh", "paper_2405_16267_b300/csrc/nspace.cuh",
                "paper_2405_16267_b300/csrc/common.cuh"]


# The same for the tensor-core softmax pass (60000-row capture scaled to 500000 rows).
TC_TRAFFIC = {"sources_sha256": "5fd8133572aac453629a0bbeb886b020eee01c6c0283157b829d31e029c909dc", "bytes_per_launch": 2.5062e+09,
              "capture": "profiles/k_fused_pass_tc2_sparse_softmax_500000x2000x10_bf16.md"}
TC_SOURCES = ["paper_2405_16267_b300/csrc/mc_tc2.cuh", "paper_2405_16267_b300/csrc/mc_tc.cuh",
              "paper_2405_16267_b300/csrc/nspace.cuh", "paper_2405_16267_b300/csrc/common.cuh",
              "paper_2405_16267_b300/csrc/pass.cuh"]

# The same kernel on the sparsity path (10 logistic instances as its columns; 60000-row
# capture scaled to 500000 rows).
PATH_TRAFFIC = {"sources_sha256": "5fd8133572aac453629a0bbeb886b020eee01c6c0283157b829d31e029c909dc", "bytes_per_launch": 2.4615e+09,
                "capture": "profiles/k_fused_pass_tc_logistic_path10_500000x2000_bf16.md"}


def pass_sources_sha256(sources=None):
    import hashlib
    h = hashlib.sha256()
    for rel in (PASS_SOURCES if sources is None else sources):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def pass_traffic(guard=None, sources=None):
    guard = PASS_TRAFFIC if guard is None else guard
    try:
        if pass_sources_sha256(sources) == guard["sources_sha256"]:
            return guard["bytes_per_launch"]
    except OSError:
        pass
    return None


def reduce_max(x, device):
    """Max of a per-rank scalar over all ranks (the timing rule: slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, steps, t_max):
    """Whole-job throughput: every rank runs `steps` iterations of its own replica."""
    return world * steps / t_max


# ----------------------------------------------------------------------------- GPU arm

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def run_gpu(args, rank, world):
    import torch
    from paper_2405_16267_b300 import bicadmm as bc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = dict(WORKLOAD)
    if args.m:
        wl["m"] = args.m
    A_np, b_np, _ = generate(wl)
    A_pin = torch.from_numpy(A_np).pin_memory()
    b_pin = torch.from_numpy(b_np).pin_memory()
    del A_np
    stream = torch.cuda.current_stream(dev)
    params = dict(loss=bc.LOSS_LOGISTIC, precision=bc.PREC_FP32, N=wl["N"], M=wl["M"],
                  kappa=wl["kappa"], gamma=wl["gamma"], rho_c=wl["rho"],
                  pass_rows=args.pass_rows, pass_stages=args.pass_stages, inner_iters=args.inner)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- device-resident timing
    s = bc.Solver(A_pin, b_pin, stream=stream, **params)
    s.step(args.warmup, info=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    time.sleep(0.15)
    bc.set_profiling(s.h, True)
    info0 = s.step(0)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps, info=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    pass_ms, pass_launches = bc.get_pass_time(s.h)
    info1 = s.step(0)
    launches = info1.kernel_launches - info0.kernel_launches
    s.close()

    # ---- end-to-end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        p = bc.default_params(loss=params["loss"], precision=params["precision"], m=wl["m"],
                              n=wl["n"], N_shards=wl["N"], M_blocks=wl["M"], kappa=wl["kappa"],
                              gamma=wl["gamma"], rho_c=wl["rho"], inner_iters=args.inner)
        h = bc.create(p, stream)
        bc.setup(h, A_pin, b_pin)
        bc.step(h, args.steps, info=False)
        x = bc.get_x(h, wl["n"])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        bc.destroy(h)
        barrier()
        e2e_s = t1 - t0
        h2d = A_pin.numel() * A_pin.element_size() + b_pin.numel() * b_pin.element_size()
        d2h = x.nbytes
        e2e = {"value": args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "seconds": e2e_s, "includes": "create+setup(H2D A,b; Gram; Cholesky; inverse)+K iterations+get_x"}

    # max over ranks
    t_local = ms / 1000.0
    t_max = reduce_max(t_local, dev) if world > 1 else t_local
    if e2e and world > 1:
        e2e["value"] = aggregate_value(world, args.steps, reduce_max(e2e["seconds"], dev))

    hbm, peak_kind = peaks()
    m, n = wl["m"], wl["n"]
    pass_bytes = m * n * 4 + 4 * m * 4  # A once + b, nu read, omega, nu written (FP32)
    avg_pass_s = pass_ms / 1000.0 / max(pass_launches, 1)
    achieved = pass_bytes / avg_pass_s / 1e9
    result = {
        "metric": METRIC, "value": aggregate_value(world, args.steps, t_max), "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; shapes and distributions of the paper-style logistic workload)",
        "config": config_dict(wl, {"inner_iters": args.inner}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": pass_traffic() if wl["m"] == WORKLOAD["m"] else None,
                     "kernel": "k_fused_pass", "peak_kind": peak_kind + " copy bandwidth",
                     "algorithmic_bytes_per_launch": pass_bytes,
                     "avg_launch_ms": avg_pass_s * 1e3, "launches_timed": pass_launches},
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    return result


# ----------------------------------------------------------------------------- softmax

SOFTMAX = dict(name="sparse_softmax_500000x2000x10_bf16", m=500000, n=2000, K=10, nnz=500, N=32,
               M=4, kappa=500, rho=1.0, gamma=10.0, seed=0)


def generate_softmax(wl, rows=None):
    """Seeded FP32 A rows and class labels of the softmax workload (shard by shard)."""
    m = wl["m"]
    r0, r1 = (0, m) if rows is None else rows
    from concurrent.futures import ThreadPoolExecutor
    pieces = [(max(a, r0), min(b_, r1)) for (a, b_) in synth.split_ranges(m, wl["N"])
              if max(a, r0) < min(b_, r1)]
    out_A = np.empty((r1 - r0, wl["n"]), dtype=np.float32)
    out_b = np.empty(r1 - r0)

    def job(rng):
        lo, hi = rng
        P = synth.sparse_softmax(m=m, n=wl["n"], K=wl["K"], nnz=wl["nnz"], N=wl["N"], M=wl["M"],
                                 kappa=wl["kappa"], seed=wl["seed"], rows=(lo, hi))
        out_A[lo - r0:hi - r0] = P.A
        out_b[lo - r0:hi - r0] = P.b

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        list(ex.map(job, pieces))
    return out_A, out_b


def run_softmax(args, rank, world):
    """Sparse softmax regression, 10 classes, A 500000 x 2000 stored in BF16 (FP32 products on
    the tensor cores), N = 32 shards, M = 4 blocks, entrywise kappa = 500.  A step is one
    outer iteration (x-update, tensor-core A pass with the softmax prox, consensus, duals)."""
    import torch
    from paper_2405_16267_b300 import bicadmm as bc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = dict(SOFTMAX)
    if args.m:
        wl["m"] = args.m
    t_gen = time.perf_counter()
    A_np, b_np = generate_softmax(wl)
    A_pin = torch.from_numpy(A_np).to(torch.bfloat16).pin_memory()  # BF16 host copy
    b_pin = torch.from_numpy(b_np).pin_memory()
    del A_np
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream(dev)
    params = dict(loss=bc.LOSS_SOFTMAX, precision=bc.PREC_BF16, N=wl["N"], M=wl["M"], K=wl["K"],
                  kappa=wl["kappa"], gamma=wl["gamma"], rho_c=wl["rho"], pass_rows=args.pass_rows,
                  inner_iters=args.inner)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    s = bc.Solver(A_pin, b_pin, stream=stream, **params)
    s.step(args.warmup, info=False)
    torch.cuda.synchronize()
    # live per-kernel times on a few extra steps (events around every launch)
    bc.set_profiling(s.h, 2)
    s.step(min(20, args.steps), info=False)
    kt = bc.get_kernel_times(s.h)
    clocks = ClockSampler(local)
    time.sleep(0.15)
    bc.set_profiling(s.h, 1)
    info0 = s.step(0)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps, info=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    pass_ms, pass_launches = bc.get_pass_time(s.h)
    info1 = s.step(0)
    launches = info1.kernel_launches - info0.kernel_launches
    s.close()

    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        p = bc.default_params(loss=params["loss"], precision=params["precision"], m=wl["m"],
                              n=wl["n"], K=wl["K"], N_shards=wl["N"], M_blocks=wl["M"],
                              kappa=wl["kappa"], gamma=wl["gamma"], rho_c=wl["rho"],
                              inner_iters=args.inner)
        h = bc.create(p, stream)
        bc.setup(h, A_pin, b_pin)
        bc.step(h, args.steps, info=False)
        x = bc.get_x(h, wl["n"] * wl["K"])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        bc.destroy(h)
        barrier()
        e2e_s = t1 - t0
        h2d = A_pin.numel() * A_pin.element_size() + b_pin.numel() * b_pin.element_size()
        e2e = {"value": args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": x.nbytes / args.steps, "seconds": e2e_s,
               "includes": "create+setup(H2D of BF16 A and b; Gram; Cholesky; inverse)+K iterations+get_x"}

    t_local = ms / 1000.0
    t_max = reduce_max(t_local, dev) if world > 1 else t_local
    if e2e and world > 1:
        e2e["value"] = aggregate_value(world, args.steps, reduce_max(e2e["seconds"], dev))
    hbm, peak_kind = peaks()
    m, n, K = wl["m"], wl["n"], wl["K"]
    # A once in BF16 + labels + omega and nu (K floats each) read and written
    pass_bytes = m * n * 2 + m * (4 + 16 * K)
    avg_pass_s = pass_ms / 1000.0 / max(pass_launches, 1)
    achieved = pass_bytes / avg_pass_s / 1e9
    cfg = {"workload": wl["name"], "m": m, "n": n, "K": K, "N_shards": wl["N"], "M_blocks": wl["M"],
           "kappa": wl["kappa"], "rho": wl["rho"], "gamma": wl["gamma"], "loss": "softmax",
           "A_dtype": "bf16", "inner_iters": args.inner,
           "l2": "inputs larger than L2 (A is %.1f GB)" % (m * n * 2 / 1e9), "parallelism": "replicas"}
    return {
        "metric": METRIC, "value": aggregate_value(world, args.steps, t_max), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded; Gaussian A, 500-entry planted W*, Gumbel-argmax labels)",
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": pass_traffic(TC_TRAFFIC, TC_SOURCES) if wl["m"] == SOFTMAX["m"] else None,
                     "kernel": "k_fused_pass_tc2",
                     "peak_kind": peak_kind + " copy bandwidth",
                     "algorithmic_bytes_per_launch": pass_bytes, "avg_launch_ms": avg_pass_s * 1e3,
                     "launches_timed": pass_launches},
        "live_kernel_ms": {k: (a / b if b else None) for k, (a, b) in kt.items()},
        "clocks": clk, "gpu_launches": int(launches), "e2e": e2e, "input_generation_s": t_gen,
    }


def softmax_leg(args):
    """The softmax workload's figures (tensor-core pass), measured in the default run so they
    appear beside the headline: its own value, roofline of k_fused_pass_tc2 and end to end."""
    import copy
    a = copy.copy(args)
    a.steps = min(args.steps, 300)
    a.warmup = max(args.warmup, 3)
    a.pass_rows = 0
    a.inner = 1
    r = run_softmax(a, 0, 1)
    keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config",
            "roofline", "e2e", "gpu_launches", "clocks", "live_kernel_ms")
    return {k: r[k] for k in keep if k in r}


PATH = dict(name="logistic_path10_500000x2000_bf16", m=500000, n=2000, nnz=50, corr=0.3, noise=0.5,
            N=32, M=4, kappa=50, rho=0.5, gamma=10.0, seed=0,
            kappas=[20, 35, 50, 75, 100, 150, 200, 300, 500, 800])


def run_path(args, rank, world):
    """A sparsity path: 10 instances of sparse logistic regression (A 500000 x 2000, Toeplitz
    feature correlation, 50-sparse model, stored in BF16), kappa from 20 to 800, solved
    together on one copy of A (bicadmm_create_path): each inner sweep's products for all 10
    are one tensor-core pass (A X and A'D as skinny GEMMs).  A step advances every instance
    by one outer iteration.  The same data solved by one single-kappa handle gives the
    per-instance cost without sharing."""
    import torch
    from paper_2405_16267_b300 import bicadmm as bc
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = dict(PATH)
    if args.m:
        wl["m"] = args.m
    A_np, b_np, _ = generate(wl)
    A_pin = torch.from_numpy(A_np).to(torch.bfloat16).pin_memory()
    b_pin = torch.from_numpy(b_np).pin_memory()
    del A_np
    stream = torch.cuda.current_stream(dev)
    R = len(wl["kappas"])
    common = dict(loss=bc.LOSS_LOGISTIC, N=wl["N"], M=wl["M"], gamma=wl["gamma"], rho_c=wl["rho"],
                  precision=bc.PREC_BF16, stream=stream)

    def timed(step, steps):
        step(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    clocks = ClockSampler(local)
    time.sleep(0.15)
    ps = bc.PathSolver(A_pin, b_pin, kappas=wl["kappas"], **common)
    bc.set_profiling(ps.h, 1)
    info0 = ps.step(0)
    ms = timed(lambda k: ps.step(k, info=False), args.steps)
    pass_ms, pass_launches = bc.get_pass_time(ps.h)
    info1 = ps.step(0)
    launches = info1.kernel_launches - info0.kernel_launches
    ps.close()
    one = bc.Solver(A_pin, b_pin, kappa=wl["kappa"], **common)
    ms_one = timed(lambda k: one.step(k, info=False), args.steps)
    one.close()
    clk = clocks.stop()
    hbm, peak_kind = peaks()
    m, n = wl["m"], wl["n"]
    pass_bytes = m * n * 2 + m * (4 + 16 * R)  # A once (BF16), b, omega and nu (R floats) in and out
    avg_pass_s = pass_ms / 1000.0 / max(pass_launches, 1)
    achieved = pass_bytes / avg_pass_s / 1e9
    per_step = ms / args.steps
    return {
        "metric": METRIC + " (every instance of the path)", "value": args.steps / (ms / 1000.0),
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic (seeded; Toeplitz-correlated A, planted 50-sparse model)",
        "config": {"workload": wl["name"], "m": m, "n": n, "N_shards": wl["N"], "M_blocks": wl["M"],
                   "kappas": wl["kappas"], "instances": R, "rho": wl["rho"], "gamma": wl["gamma"],
                   "loss": "logistic", "A_dtype": "bf16",
                   "l2": "inputs larger than L2 (A is %.1f GB)" % (m * n * 2 / 1e9)},
        "instance_iters_per_s": R * args.steps / (ms / 1000.0),
        "single_kappa_handle": {"ms_per_step": ms_one / args.steps,
                                "iters_per_s": args.steps / (ms_one / 1000.0)},
        "speedup_vs_separate_handles": R * (ms_one / args.steps) / per_step,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": pass_traffic(PATH_TRAFFIC, TC_SOURCES) if m == PATH["m"] else None,
                     "kernel": "k_fused_pass_tc2",
                     "peak_kind": peak_kind + " copy bandwidth",
                     "algorithmic_bytes_per_launch": pass_bytes, "avg_launch_ms": avg_pass_s * 1e3,
                     "launches_timed": pass_launches},
        "clocks": clk, "gpu_launches": int(launches),
    }


def path_leg(args):
    """The sparsity-path workload's figures (one tensor-core pass for 10 instances), measured in
    the default run: its value, per-instance rate, speedup over separate handles, roofline."""
    import copy
    a = copy.copy(args)
    a.steps = min(args.steps, 100)
    a.warmup = max(args.warmup, 3)
    r = run_path(a, 0, 1)
    keep = ("metric", "value", "unit", "steps", "ms_per_step", "config", "instance_iters_per_s",
            "single_kappa_handle", "speedup_vs_separate_handles", "roofline", "gpu_launches")
    return {k: r[k] for k in keep if k in r}


def run_oracle_softmax(wl, steps, budget_s=30.0):
    """The FP64 oracle on shard 0 of the softmax workload (BF16-rounded A, as the GPU path
    sees it); one full iteration extrapolated as N times one shard's iteration."""
    from oracle import bicadmm_ref as ref
    r0, r1 = synth.split_ranges(wl["m"], wl["N"])[0]
    A, b = generate_softmax(wl, rows=(r0, r1))
    A = synth.round_to_bf16(A)
    o = ref.BiCADMM(A, b, ref.LOSS_SOFTMAX, 1, wl["M"], wl["kappa"], gamma=wl["gamma"],
                    rho_c=wl["rho"], K=wl["K"], n_shards_total=wl["N"])
    o.iterate(1)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        o.iterate(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = (time.perf_counter() - t0) / done
    sample = ("shard 0 of %d (%d x %d, K=%d, FP64 on the BF16-rounded A) with M=%d blocks: %d outer "
              "iterations timed, %.3f s each; full iteration extrapolated as %d x that"
              % (wl["N"], r1 - r0, wl["n"], wl["K"], wl["M"], done, dt, wl["N"]))
    return {"value": 1.0 / (wl["N"] * dt), "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": sample, "steps_timed": done}


# ----------------------------------------------------------------------------- batch

def run_batch(args, rank, world):
    """Batched workload: args.batch uneven instances (m log-uniform in [1e3, 5e4], n
    log-uniform in [100, 4000], kappa 1-5 % of n, 4-16 shards, squared / squared-hinge loss,
    FP32), all advanced by one launch per kernel kind per iteration (CUDA graph, autotuned
    panel tiling).  A step is one outer iteration of every instance."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2405_16267_b300 import bicadmm as bc
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    specs = synth.batch_instance_specs(count=args.batch)
    prec = bc.PREC_BF16 if args.precision == "bf16" else bc.PREC_FP32
    a_es = 2 if args.precision == "bf16" else 4
    stream = torch.cuda.Stream()
    solvers, a_bytes, rows = [], 0, 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        for P in ex.map(synth.batch_instance, specs):
            with torch.cuda.stream(stream):
                solvers.append(bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa,
                                         gamma=P.gamma, rho_c=P.rho, precision=prec,
                                         stream=stream))
            a_bytes += P.m * P.n * a_es + 16 * P.m
            rows += P.m
    setup_s = time.perf_counter() - t0
    b = bc.batch_create(solvers, stream=stream, flags=bc.BATCH_GRAPH | bc.BATCH_AUTOTUNE)
    warm = max(args.warmup, 80)  # the autotuner spends the first iterations (2 per candidate tiling)
    bc.batch_step(b, warm)
    stream.synchronize()
    tiling = bc.batch_tiling(b)
    clocks = ClockSampler(local)
    time.sleep(0.15)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = bc.batch_step(b, 0)
    e0.record(stream)
    l1 = bc.batch_step(b, args.steps)
    e1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    bc.batch_destroy(b)
    # the same instances stepped one handle at a time on the same stream
    seq_steps = max(3, min(args.steps, 20))
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(seq_steps):
        for s in solvers:
            s.step(1, info=False)
    e3.record(stream)
    stream.synchronize()
    seq_ms = e2.elapsed_time(e3) / seq_steps
    for s in solvers:
        s.close()
    hbm, peak_kind = peaks()
    per_iter_s = ms / 1000.0 / args.steps
    achieved = a_bytes / per_iter_s / 1e9
    return {
        "metric": "batched ADMM iters/s (one iteration of every instance)",
        "value": aggregate_value(world, args.steps, ms / 1000.0), "unit": "batch iters/s",
        "instance_iters_per_s": args.batch * args.steps / (ms / 1000.0),
        "n_gpus": world, "steps": args.steps, "warmup": warm, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if args.precision == "bf16" else "f32", "data": "synthetic (seeded)",
        "config": {"workload": "batch%d_uneven_linear_sqhinge_%s" % (args.batch, args.precision),
                   "instances": args.batch, "rows_total": rows, "A_bytes": a_bytes,
                   "graph": True, "autotuned_tiling": {"stage_kb": tiling[0], "stages": tiling[1]},
                   "l2": "inputs larger than L2 (%.1f GB)" % (a_bytes / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None,
                     "note": "whole batched iteration (all kernels) against the A bytes + row state",
                     "peak_kind": peak_kind + " copy bandwidth"},
        "sequential_handles_ms_per_step": seq_ms,
        "batch_speedup_vs_sequential": seq_ms / (ms / args.steps),
        "setup_s": setup_s, "clocks": clk, "gpu_launches": int(l1 - l0),
    }


def batch_leg(args):
    """The batched workload's figures (256 uneven FP32 instances, autotuned tiling, CUDA
    graph), measured in the default run: its value, per-instance rate, whole-iteration
    roofline and speedup over the same handles stepped one at a time."""
    import copy
    a = copy.copy(args)
    a.steps = min(args.steps, 50)
    a.warmup = max(args.warmup, 3)
    a.batch = 256
    a.precision = "fp32"
    r = run_batch(a, 0, 1)
    keep = ("metric", "value", "unit", "steps", "ms_per_step", "dtype", "config",
            "instance_iters_per_s", "roofline", "batch_speedup_vs_sequential", "gpu_launches",
            "clocks")
    return {k: r[k] for k in keep if k in r}


# ----------------------------------------------------------------------------- serve

def run_serve(args, rank, world):
    """Serving: a Poisson stream (args.rate per second) of args.requests solves of mixed
    loss and size (m log-uniform [1e3, 2e5], n log-uniform [100, 1e4], kappa 1-5 % of n,
    FP32), inputs drawn on the device beforehand; the serving loop admits them under a
    150 GB budget with continuous batching.  Latency = completion - arrival."""
    import torch
    from paper_2405_16267_b300 import bicadmm as bc
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    specs = synth.serve_request_specs(count=args.requests, rate=args.rate)
    t_gen = time.perf_counter()
    data = [synth.device_request(sp) for sp in specs]
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    prec = bc.PREC_BF16 if args.precision == "bf16" else bc.PREC_FP32
    a_bytes = sum(sp["m"] * sp["n"] * (2 if args.precision == "bf16" else 4) for sp in specs)
    clocks = ClockSampler(local)
    with bc.Server(hbm_budget_bytes=150 << 30, max_active=64, iters_per_round=10,
                   precision=prec, use_graph=True, polish=True) as srv:
        t0 = srv.clock() + 0.05
        ids = [srv.submit(A, b, arrival=t0 + sp["arrival"], loss=sp["loss"],
                          precision=prec, N_shards=sp["N"], M_blocks=sp["M"],
                          kappa=sp["kappa"], gamma=10.0, rho_c=1.0, max_iters=args.serve_iters,
                          tol_rel=1e-6)
               for sp, (A, b) in zip(specs, data)]
        srv.run()
        res = [srv.result(i) for i in ids]
        st = srv.stats()
        tim = [srv.timing(i) for i, r in zip(ids, res) if r["status"] == 0]
        prof = srv.timing(-1)
    clk = clocks.stop()
    ok = [r for r in res if r["status"] == 0]
    lat = np.array([r["done"] - r["arrival"] for r in ok])
    wait = np.array([r["admitted"] - r["arrival"] for r in ok])

    def pct(v):
        v = np.asarray(v)
        return {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}
    # where a request's time goes: queued, its own setup, iterating in batched rounds (shared
    # with the others), and retirement (objective, polish, copy-out)
    breakdown = {"queue_s": pct([t["admitted"] - t["arrival"] for t in tim]),
                 "setup_s": pct([t["setup_done"] - t["admitted"] for t in tim]),
                 "rounds_s": pct([t["retiring"] - t["setup_done"] for t in tim]),
                 "retire_s": pct([t["done"] - t["retiring"] for t in tim]),
                 "rounds_per_request": pct([t["rounds"] for t in tim])}
    span = max(r["done"] for r in res) - min(r["arrival"] for r in res)
    return {
        "metric": "solves/s (serving, continuous batching)", "value": len(ok) / span,
        "unit": "solves/s", "n_gpus": world, "steps": len(res), "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if args.precision == "bf16" else "f32",
        "data": "synthetic (seeded, drawn on the device)",
        "config": {"workload": "serve_poisson%d_mixed_%s" % (int(args.rate), args.precision),
                   "requests": len(res), "arrival_rate_per_s": args.rate,
                   "offered_A_bytes": a_bytes, "hbm_budget_bytes": 150 << 30,
                   "iters_per_request_cap": args.serve_iters, "tol_rel": 1e-6,
                   "iters_per_round": 10},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "completed": len(ok), "failed": len(res) - len(ok),
        "converged": int(sum(r["info"].converged for r in ok)),
        "request_breakdown": breakdown,
        "server_loop_s": {k: prof[k] for k in ("rebuild_s", "round_wait_s", "admit_s", "retire_s")},
        "batch_rebuilds": int(prof["rebuilds"]),
        "server": st, "input_generation_s": t_gen, "clocks": clk,
        "gpu_launches": int(st["launches"]),
    }


# ----------------------------------------------------------------------------- time to tol

TABLE1 = dict(m=100000, n=2000, sparsity=0.9, noise=0.01, N=4, M=4, rho=1.0, gamma=10.0, seed=0)
TABLE1_PAPER_S = 1.1  # Table 1: m = 1e5, n = 2k, s_l = 0.9 (RTX 4070 + i7-13700; tolerance unstated)


def run_time_to_tol(stream, tol=1e-6):
    """Time to max(p_rel, d_rel, b_rel, i_rel) <= tol on the paper's Table-1 setting, for the
    plain FP64 path and the FP32 path on the same inputs (A on the device before timing)."""
    import torch
    from paper_2405_16267_b300 import bicadmm as bc
    P = synth.table1_sls(**TABLE1)
    A64 = torch.from_numpy(P.A).cuda()
    A32 = A64.float()
    b64 = torch.from_numpy(P.b).cuda()
    truth = set(np.flatnonzero(P.x_star).tolist())
    out = {"workload": P.name, "tol_rel": tol, "N_shards": P.N, "M_blocks": P.M, "kappa": P.kappa,
           "check_every": 5}
    for name, prec in (("fp64", bc.PREC_FP64), ("fp32", bc.PREC_FP32)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = bc.Solver(A64 if prec == bc.PREC_FP64 else A32, b64, loss=P.loss, N=P.N, M=P.M,
                      kappa=P.kappa, gamma=P.gamma, rho_c=P.rho, precision=prec, tol_rel=tol,
                      check_every=5, max_iters=5000, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        info = s.solve()
        t2 = time.perf_counter()
        x, supp = bc.get_x(s.h, P.n, polished=True, with_support=True, kappa=P.kappa)
        t3 = time.perf_counter()
        s.close()
        out[name] = {"setup_s": t1 - t0, "solve_s": t2 - t1, "polish_s": t3 - t2,
                     "iters": int(info.iters), "converged": bool(info.converged),
                     "support_recovered": set(supp.tolist()) == truth,
                     "rel_err_polished_vs_planted": float(np.linalg.norm(x - P.x_star) / np.linalg.norm(P.x_star))}
    out["solve_speedup_fp32_vs_fp64"] = out["fp64"]["solve_s"] / out["fp32"]["solve_s"]
    # The served form: the same problem through the serving loop (continuous batching) in
    # FP32 and BF16 storage, alone and in a mix with three other Table-1 instances arriving
    # together; time = result ready minus arrival (setup, rounds with tolerance checks and the
    # polish included), against the plain FP64 path's setup + solve + polish.
    x64 = None
    with bc.Solver(A64, b64, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma, rho_c=P.rho,
                   precision=bc.PREC_FP64, tol_rel=tol, check_every=5, max_iters=5000, stream=stream) as s:
        s.solve()
        x64 = bc.get_x(s.h, P.n, polished=True)
    fp64_total = out["fp64"]["setup_s"] + out["fp64"]["solve_s"] + out["fp64"]["polish_s"]
    others = [synth.table1_sls(**dict(TABLE1, seed=TABLE1["seed"] + q)) for q in (1, 2, 3)]
    A_others = [torch.from_numpy(Q.A).float().cuda() for Q in others]
    b_others = [torch.from_numpy(Q.b).cuda() for Q in others]
    for name, prec in (("served_fp32", bc.PREC_FP32), ("served_bf16", bc.PREC_BF16)):
        entry = {}
        for mix in (False, True):
            with bc.Server(hbm_budget_bytes=40 << 30, max_active=8, iters_per_round=10,
                           precision=prec, polish=True) as srv:
                common = dict(gamma=P.gamma, rho_c=P.rho, tol_rel=tol, check_every=5, max_iters=5000,
                              precision=prec)
                torch.cuda.synchronize()
                t0 = srv.clock()
                rid = srv.submit(A32, b64, arrival=t0, loss=P.loss, N_shards=P.N, M_blocks=P.M,
                                 kappa=P.kappa, **common)
                mates = []
                if mix:
                    for Q, Aq, bq in zip(others, A_others, b_others):
                        mates.append(srv.submit(Aq, bq, arrival=t0, loss=Q.loss, N_shards=Q.N,
                                                M_blocks=Q.M, kappa=Q.kappa, **common))
                srv.run()
                r = srv.result(rid)
                rm = [srv.result(q) for q in mates]
            x = r["x"]
            e = {"time_s": r["done"] - r["arrival"], "iters": int(r["info"].iters),
                 "converged": bool(r["info"].converged),
                 "support_recovered": set(r["support"].tolist()) == truth,
                 "rel_diff_vs_fp64_polished": float(np.linalg.norm(x - x64) / np.linalg.norm(x64))}
            if mix:
                e["all_four_done_s"] = max([r["done"]] + [q["done"] for q in rm]) - r["arrival"]
                e["all_converged"] = bool(r["info"].converged) and all(bool(q["info"].converged) for q in rm)
            entry["in_mix_of_4" if mix else "alone"] = e
        entry["speedup_vs_fp64_alone"] = fp64_total / entry["alone"]["time_s"]
        out[name] = entry
    out["paper_table1_s"] = {"value": TABLE1_PAPER_S, "hardware": "RTX 4070 + i7-13700, PyTorch 2.3",
                             "note": "context only: other machine, tolerance unstated"}
    return out


# ----------------------------------------------------------------------------- CPU oracle

def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([d.get("num_threads", 1) for d in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


def run_oracle_sample(wl, steps, warmup, budget_s=90.0):
    """Time the FP64 oracle on shard 0 of the workload (a bounded sample) and extrapolate
    one outer iteration of the whole workload as N times one sampled shard iteration."""
    from oracle import bicadmm_ref as ref
    r0, r1 = synth.split_ranges(wl["m"], wl["N"])[0]
    A, b, _ = generate(wl, rows=(r0, r1))
    A = A.astype(np.float64)
    o = ref.BiCADMM(A, b, ref.LOSS_LOGISTIC, 1, wl["M"], wl["kappa"], gamma=wl["gamma"],
                    rho_c=wl["rho"])
    o.iterate(max(1, min(warmup, 2)))
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        o.iterate(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = (time.perf_counter() - t0) / done
    value = 1.0 / (wl["N"] * dt)
    sample = ("shard 0 of %d (%d x %d rows x cols, FP64) with M=%d blocks: %d outer iterations "
              "timed, %.3f s each; full iteration extrapolated as %d x that"
              % (wl["N"], r1 - r0, wl["n"], wl["M"], done, dt, wl["N"]))
    return {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": sample, "steps_timed": done, "seconds_per_sample_step": dt,
            "seconds_timed": dt * done, "extrapolated": True}


def run_reference(args, rank, world):
    """The oracle arm.  A step here is what was actually timed: one outer iteration of shard
    0 (1/N of the workload's rows); steps x ms_per_step is the time spent.  `value` is the
    whole workload's iterations/s, extrapolated as N shard iterations per iteration
    (`extrapolated`, `extrapolation_factor`)."""
    if rank != 0:
        return None
    wl = dict(WORKLOAD)
    cb = run_oracle_sample(wl, args.steps, args.warmup)
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": world, "steps": cb["steps_timed"], "warmup": args.warmup,
            "ms_per_step": 1000.0 * cb["seconds_per_sample_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "step_unit": "one outer iteration of shard 0 of %d (the timed sample)" % wl["N"],
            "extrapolated": True, "extrapolation_factor": wl["N"],
            "timed_seconds": cb["seconds_timed"],
            "config": config_dict(wl), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "gpu":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    elif args.workload == "batch":
        res = run_batch(args, rank, world)
    elif args.workload == "serve":
        res = run_serve(args, rank, world)
    elif args.workload == "path":
        res = run_path(args, rank, world)
    elif args.workload == "softmax":
        res = run_softmax(args, rank, world)
        if rank == 0 and not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = run_oracle_softmax(dict(SOFTMAX), steps=10, budget_s=25.0)
    else:
        res = run_gpu(args, rank, world)
        if rank == 0 and not args.no_ttt:
            import torch
            res["time_to_tol"] = run_time_to_tol(torch.cuda.current_stream())
        if rank == 0 and not args.no_cpu_baseline and world == 1:
            res["cpu_baseline"] = run_oracle_sample(dict(WORKLOAD), steps=8, warmup=1, budget_s=20.0)
        if world == 1 and not args.no_legs and args.m is None:
            res["legs"] = {}
            for name, leg in (("softmax", softmax_leg), ("path", path_leg), ("batch", batch_leg)):
                try:
                    res["legs"][name] = leg(args)
                except Exception as exc:  # a leg never costs the headline line
                    res["legs"][name] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if world > 1 and args.impl == "gpu":
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
