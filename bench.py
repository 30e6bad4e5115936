#!/usr/bin/env python3
"""Benchmark: device-timed GFLOP/s (Eq. 1, 2*M*N*K/t) of one grouped launch
over the uneven batch -- 200,000 FP32 instances with M, N, K log-uniform on
[1, 80], all four cases, ld = rows + U{0..7} -- with its roofline fraction,
the end-to-end rate through the C ABI from pinned host memory, and the FP64
CPU oracle as the reported baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision ffma]
    python bench.py --workload uneven-c64 ...   # other batches (see WORKLOADS)
    python bench.py --impl reference ...   # the CPU oracle arm
    python bench.py --pack-ablation        # pack-step share by size (Fig. 3 on this GPU)
    python bench.py --sweep                # same-size batches M = N = K = n, every case and pipe

One step = one execution of the whole plan (one persistent kernel launch,
replayed from a CUDA graph).  The pools (about 1.3 GB) are larger than the
129 MB L2, so no flush is needed between steps.  Under torchrun each rank runs
its own copy of the batch (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "small-GEMM GFLOP/s & roofline % (uneven batch), TC split vs plain FP32 @1e-5"
WORKLOAD = ("uneven-{n}-fp32: {n} instances, M,N,K log-uniform int [1,80], NN/NT/TN/TT uniform "
            "(TN redrawn to MNK<=32768), ld=rows+U{{0..7}}, alpha,beta~U[-2,2], N(0,1), seed 2")
NOMINAL_HBM_GBS = 8000.0
# paths that route small instances to the FP32 CUDA-core kernel: name ->
# (route_k_below, route_mnk_below, route_kernel); "d": the CUDA-core part on
# the warp-direct kernel
ROUTE = {"3xbf16-k8ffma": (8, 0, 0), "3xbf16-r8": (8, 8 ** 3, 0), "3xbf16-r12": (8, 12 ** 3, 0),
         "3xbf16-r16": (8, 16 ** 3, 0), "3xbf16-r24": (8, 24 ** 3, 0), "3xbf16-r32": (8, 32 ** 3, 0)}
ROUTE.update({"3xbf16-k8d": (8, 0, 4)})
ROUTE.update({f"3xbf16-r{n}d": (8, n ** 3, 4) for n in (8, 12, 16, 20, 24, 32, 40, 48, 64)})
PRECISIONS = {"ffma": 0, "3xbf16": 1, "tf32": 2, "fp16": 3, "6xbf16": 4}
PRECISIONS.update({n: 1 for n in ROUTE})
# each path can also be forced onto one kernel family: name + "@stage"
# (stage-program kernels), name + "@stream" (warp-stream / pack-stream), for
# the tensor-core paths name + "@warp" (warp-tile kernel), for FFMA name +
# "@direct" (warp-direct kernel)
for _n in list(PRECISIONS):
    PRECISIONS[_n + "@stage"] = PRECISIONS[_n + "@stream"] = PRECISIONS[_n]
    if PRECISIONS[_n]:
        PRECISIONS[_n + "@warp"] = PRECISIONS[_n]
    else:
        PRECISIONS[_n + "@direct"] = PRECISIONS[_n]
# the FP64 batches' DFMA path, on the stage programs or the warp-direct kernel
PRECISIONS.update({"dfma": 0, "dfma@direct": 0})
KERNEL = {n: {"stage": 1, "stream": 2, "warp": 3, "direct": 4}.get(n.split("@")[1], 0) if "@" in n else 0
          for n in PRECISIONS}
ROUTE_BASE = lambda n: n.split("@")[0]

# Batches bench.py can time.  The default is the uneven FP32 batch (the
# headline); the others run the CUDA-core path of their type only:
# name -> (generator, description, default instances, dtype code, path name, tolerance)
WORKLOADS = {
    "uneven": ("uneven", WORKLOAD, 200_000, 0, None, 1e-5),
    "uniform16": ("uniform16", "uniform16-{n}: {n} FP32 NN instances of 16x16x16, ld=16, alpha=1, beta=0.5, "
                  "U[-1,1], seed 0; the pools fit L2, so launches rotate over five copies of them "
                  "(5 x 41 MB > 129 MB)", 10_000, 0, None, 1e-5),
    "fc64": ("fc64", "fc64-{n}: {n} FP64 instances, M in {{32,64}}, K,N log-uniform int [8,80], NN/TN 50/50 "
             "(TN redrawn to MNK<=32768), alpha=1, beta in {{0,1}}, U[-1,1], seed 4", 100_000, 1, "dfma", 1e-13),
    "uneven-c32": ("uneven_complex", "uneven-{n}-c32: {n} complex-float instances (CGEMM), M,N,K log-uniform "
                   "int [1,80], NN/NT/TN/TT uniform (TN redrawn to MNK<=32768), ld=rows+U{{0..7}}, alpha,beta "
                   "parts ~U[-2,2], N(0,1) parts, seed 5", 100_000, 2, "cgemm", 1e-5),
    "uneven-c64": ("uneven_complex", "uneven-{n}-c64: {n} complex-double instances (ZGEMM), M,N,K log-uniform "
                   "int [1,80], NN/NT/TN/TT uniform (TN redrawn to MNK<=32768), ld=rows+U{{0..7}}, alpha,beta "
                   "parts ~U[-2,2], N(0,1) parts, seed 5", 100_000, 3, "zgemm", 1e-13),
}
DTYPE_NAMES = {0: "f32", 1: "f64", 2: "c32", 3: "c64"}


def make_workload(name, n):
    from paper_2208_09822_gb300 import workloads as W
    gen, _, default_n, code, _, _ = WORKLOADS[name]
    n = default_n if n is None else n
    if gen == "uneven_complex":
        return W.uneven_complex(count=n, dtype=np.complex64 if code == 2 else np.complex128)
    return getattr(W, gen)(count=n)


def shard_ranges(batch, world):
    """--split shard: the contiguous instance range [i0, i1) of every rank,
    cut with shard.shard_bounds on shard.instance_cost so that the ranks get
    about the same work, with each range's flops and the element spans
    [lo, hi) of its A, B and C in the pools (what the rank copies in and
    out end to end).  The ranges cover the batch once, in order."""
    from paper_2208_09822_gb300.shard import instance_cost, shard_bounds
    cost = instance_cost(batch.M, batch.N, batch.K, batch.beta != 0, batch.esize)
    n = batch.count
    out = []
    for i0, i1 in shard_bounds(cost, world):
        def span(off, pool):
            return (int(off[i0]) if i0 < n else pool.size, int(off[i1]) if i1 < n else pool.size)
        sub = batch.select(np.arange(i0, i1))
        out.append({"i0": i0, "i1": i1, "flops": sub.flops() if i1 > i0 else 0,
                    "A": span(batch.offA, batch.A), "B": span(batch.offB, batch.B), "C": span(batch.offC, batch.C)})
    return out


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# the translation unit that holds each path's grouped kernel
KERNEL_UNITS = {"ffma": "kernels_fma.cu", "dfma": "kernels_fma.cu", "cgemm": "kernels_cplx.cu",
                "zgemm": "kernels_cplx.cu"}


def kernel_unit(precision, family=None):
    """The translation unit of a path's kernel; `family` is the plan's
    kernel_family (1 stage, 2 stream, 3 warp-tile), else the path's suffix."""
    base = ROUTE_BASE(precision)
    if family is None:
        family = KERNEL.get(precision, 0) or 1
    if base in ("ffma", "dfma"):
        return {2: "kernels_ws.cu", 4: "kernels_wd.cu"}.get(family, KERNEL_UNITS[base])
    if base in KERNEL_UNITS:
        return KERNEL_UNITS[base]
    return {2: "kernels_tc2.cu", 3: "kernels_tw.cu"}.get(family, "kernels_tc.cu")


def kernel_source_hash(precision="3xbf16", family=None):
    """Hash of the sources a path's kernel is compiled from: its translation
    unit and every header it includes (launch.h, which only declares the
    host launchers, aside), so a profile stays current while that kernel's
    code is unchanged.  A routed path hashes its CUDA-core kernel's sources
    too: its launches run both."""
    csrc = os.path.join(ROOT, "paper_2208_09822_gb300", "csrc")
    seen, todo = set(), [kernel_unit(precision, family)]
    if ROUTE_BASE(precision) in ROUTE:
        todo.append("kernels_wd.cu" if ROUTE[ROUTE_BASE(precision)][2] == 4 else KERNEL_UNITS["ffma"])
    while todo:
        f = todo.pop()
        if f in seen or f == "launch.h" or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            todo += re.findall(r'^#include "([^"/]+)"', fh.read(), re.M)
    h = hashlib.sha256()
    for f in sorted(seen):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profile_traffic(precision, workload="uneven", count=200_000, family=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"grouped_{precision}_{workload}{count // 1000}k.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    kv = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_source_hash") != kernel_source_hash(precision, family):
        return None
    try:
        return float(kv["dram_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sms:
            return None
        return {"sm_mhz": float(np.median(sms)), "sm_max_mhz": float(max(maxes)),
                "reasons": sorted(reasons), "samples": len(sms)}


def cpu_baseline_leg(batch, gpu_results, min_seconds, tol=1e-5):
    """The CPU-baseline leg: time the FP64 oracle over the whole batch
    (repeated until min_seconds), and use its result to measure the error of
    each path's first launch."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from gpu_util import errors
    run = oracle.cgemm_batch if batch.is_complex else oracle.gemm_batch
    flops = batch.flops()
    t0 = time.perf_counter()
    reps = 0
    while True:
        ref, _ = run(batch)
        reps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    cpu = {"value": flops * reps / dt / 1e9, "unit": "GFLOP/s", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": f"the whole batch, {reps} pass(es) in {dt:.1f} s, FP64 triple loop"}
    errs = {}
    for name, res in gpu_results.items():
        e = errors(batch, res, ref)
        errs[name] = {k: e[k] for k in ("eps_batch", "eps_inst_max", "eps_inst_median", "eps_inst_rms")}
        errs[name][f"within_{tol:g}"] = e["eps_batch"] <= tol
    return cpu, errs


def run_reference(args):
    """CPU oracle arm: FP64 triple loop over the same batch on the host cores."""
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    import oracle
    batch = make_workload(args.workload, args.instances)
    run = oracle.cgemm_batch if batch.is_complex else oracle.gemm_batch
    # one step = the oracle over a bounded sample of the batch (every 8th instance)
    sample = batch.select(np.arange(0, batch.count, 8))
    flops = sample.flops()
    for _ in range(args.warmup):
        run(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(sample)
    dt = time.perf_counter() - t0
    value = flops * args.steps / dt / 1e9
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1].format(n=batch.count),
                   "sample": f"every 8th instance ({sample.count} instances, "
                                                   f"{flops / 1e9:.3f} GFLOP) per step"},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"every 8th instance of the batch ({sample.count}), FP64 triple loop"},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_pack_ablation(args):
    """The GPU analogue of Fig. 3 (the share of a traditional GEMM's time spent
    in its pack step).  For same-size FP32 batches (M = N = K = n, 4096
    instances, tight ld, alpha = 1.25, beta = -0.75, each case) time: the
    library's grouped GEMM on the operands where they are (no pack), the pack
    step (op(A), op(B) copied into tight NN copies; one kernel), and the same
    grouped GEMM on the packed copies.  share = pack / (pack + packed GEMM);
    slowdown = (pack + packed GEMM) / no-pack.  CUDA events on the launch
    stream, 3 untimed runs then `--steps` (at most 50) timed runs of each."""
    import torch
    torch.cuda.set_device(0)
    from paper_2208_09822_gb300 import build as B
    B.build()
    from paper_2208_09822_gb300 import iaat
    from paper_2208_09822_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    reps = max(1, min(args.steps, 50))

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rows = []
    launches = 0
    for case in ("NN", "NT", "TN", "TT"):
        for n in (1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 80):
            if not W.in_domain(n, n, n, *W.TRANS_CASES[case]):
                continue
            b = W.sweep(case, (n, n, n), count=4096)
            tA = torch.from_numpy(b.A).to(dev)
            tB = torch.from_numpy(b.B).to(dev)
            tC = torch.from_numpy(b.C).to(dev)
            descs = iaat.descs_for_pools(b, tA.data_ptr(), tB.data_ptr(), tC.data_ptr())
            direct = iaat.iaat_plan_create(descs, iaat.IAAT_F32)
            pk = iaat.iaat_pack_create(descs, iaat.IAAT_F32)
            packed = iaat.iaat_plan_create(pk.packed, iaat.IAAT_F32)
            t_direct = timed(lambda: iaat.iaat_gemm_grouped(direct, stream))
            t_pack = timed(lambda: iaat.iaat_pack_run(pk, stream))
            t_packed = timed(lambda: iaat.iaat_gemm_grouped(packed, stream))
            iaat.iaat_plan_check(direct, stream)
            iaat.iaat_plan_check(packed, stream)
            launches += 3 * (reps + 3)
            rows.append({"case": case, "n": n, "no_pack_us": t_direct * 1e3, "pack_us": t_pack * 1e3,
                         "gemm_on_packed_us": t_packed * 1e3, "pack_share": t_pack / (t_pack + t_packed),
                         "slowdown_vs_no_pack": (t_pack + t_packed) / t_direct,
                         "pack_GBs": pk.bytes_moved / (t_pack * 1e-3) / 1e9})
            for x in (direct, packed, pk):
                x.destroy()
    print(json.dumps({"metric": "pack-step share of a packed small GEMM (GPU analogue of Fig. 3)",
                      "unit": "fraction", "dtype": "f32", "data": "synthetic", "n_gpus": 1,
                      "config": {"workload": "sweep: 4096 same-size FP32 instances per launch, M=N=K=n, "
                                             "tight ld, alpha=1.25, beta=-0.75, U[-1,1], seed 1",
                                 "reps": reps, "l2": "n <= 48 fits the 129 MB L2; no flush (an ablation)"},
                      "rows": rows, "gpu_launches": launches}), flush=True)
    return 0


def run_sweep(args):
    """Same-size batches on the M = N = K diagonal of the sweep sizes (4096
    instances per launch, tight ld, alpha = 1.25, beta = -0.75, U[-1,1],
    seed 1), every case, on the FFMA, 3xBF16 and DFMA paths: device time per
    launch (CUDA events, 3 untimed then `--steps` (at most 20) timed launches
    back to back), GFLOP/s (Eq. 1) and the fraction of the roofline, the slower
    of the algorithmic bytes at the measured copy bandwidth and the flops at
    the path's pipe peak (measured FFMA / DFMA rates, the measured BF16 burst
    rate for the useful 2*M*N*K of 3xBF16)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2208_09822_gb300 import build as B
    B.build()
    from paper_2208_09822_gb300 import iaat
    from paper_2208_09822_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    reps = max(1, min(args.steps, 20))
    peaks, peak_kind = measured_peaks()
    pipe = {"ffma": iaat.iaat_fma_peak(iaat.IAAT_F32), "dfma": iaat.iaat_fma_peak(iaat.IAAT_F64),
            "3xbf16": peaks["bf16_tflops"] * 1e3}
    rows, launches = [], 0
    for case in ("NN", "NT", "TN", "TT"):
        for n in (1, 2, 4, 8, 16, 32, 48, 64, 80):
            if not W.in_domain(n, n, n, *W.TRANS_CASES[case]):
                continue
            for dtype, paths in ((np.float32, tuple(args.sweep_paths)), (np.float64, ("dfma",))):
                b = W.sweep(case, (n, n, n), dtype=dtype, count=4096)
                tA = torch.from_numpy(b.A).to(dev)
                tB = torch.from_numpy(b.B).to(dev)
                tC = torch.from_numpy(b.C).to(dev)
                descs = iaat.descs_for_pools(b, tA.data_ptr(), tB.data_ptr(), tC.data_ptr())
                for path in paths:
                    plan = iaat.iaat_plan_create(descs, iaat.IAAT_F32 if dtype == np.float32 else iaat.IAAT_F64,
                                                 PRECISIONS.get(path, 0), kernel=KERNEL.get(path, 0))
                    info = iaat.iaat_plan_info(plan)
                    with torch.cuda.stream(stream):
                        for _ in range(3):
                            iaat.iaat_gemm_grouped(plan, stream)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(stream):
                        e0.record(stream)
                        for _ in range(reps):
                            iaat.iaat_gemm_grouped(plan, stream)
                        e1.record(stream)
                    torch.cuda.synchronize()
                    iaat.iaat_plan_check(plan, stream)
                    ms = e0.elapsed_time(e1) / reps
                    launches += reps + 3
                    pk = pipe[ROUTE_BASE(path) if ROUTE_BASE(path) in pipe else "3xbf16"]
                    t_roof = max(info["algorithmic_bytes"] / (peaks["hbm_gbs"] * 1e9), info["flops"] / (pk * 1e9))
                    rows.append({"case": case, "n": n, "path": path, "us": ms * 1e3,
                                 "gflops": info["flops"] / (ms * 1e-3) / 1e9,
                                 "roofline_frac": t_roof / (ms * 1e-3),
                                 "bound": "hbm" if info["algorithmic_bytes"] / (peaks["hbm_gbs"] * 1e9)
                                 >= info["flops"] / (pk * 1e9) else path})
                    plan.destroy()
                del tA, tB, tC
    print(json.dumps({"metric": "same-size sweep GFLOP/s and roofline fraction (M = N = K)", "unit": "GFLOP/s",
                      "n_gpus": 1, "data": "synthetic",
                      "config": {"workload": "sweep diagonal: 4096 same-size instances per launch, tight ld, "
                                             "alpha=1.25, beta=-0.75, U[-1,1], seed 1", "reps": reps,
                                 "peaks": {"hbm_gbs": peaks["hbm_gbs"], "kind": peak_kind,
                                           "ffma_gflops": pipe["ffma"], "dfma_gflops": pipe["dfma"],
                                           "bf16_gflops": pipe["3xbf16"]},
                                 "l2": "n <= 48 fits the 129 MB L2; no flush"},
                      "rows": rows, "gpu_launches": launches}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="iaat", choices=["iaat", "reference"])
    ap.add_argument("--precision", default="3xbf16-r32d", choices=sorted(PRECISIONS),
                    help="the headline path: by default the tensor-core FP32 split (3xBF16) on the instances "
                         "with M*N*K >= 32^3 and K >= 8, the smaller ones on the FP32 CUDA cores (warp-direct "
                         "kernel)")
    ap.add_argument("--compare", default="ffma,ffma@direct,3xbf16,3xbf16-r16",
                    type=lambda v: [x for x in v.split(",") if x],
                    help="comma-separated paths timed beside the headline (by default plain FP32 on the stage "
                         "programs and on the warp-direct kernel, 3xBF16 for every instance, and 3xBF16 with "
                         "the small instances on the stage programs)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-chunks", type=int, default=4,
                    help="instance ranges the end-to-end leg pipelines copies and launches over")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="uneven", choices=sorted(WORKLOADS),
                    help="the batch: uneven FP32 (the headline; --precision and --compare apply), or one "
                         "timed on its CUDA-core path only (fc64, uneven-c32 = CGEMM, uneven-c64 = ZGEMM)")
    ap.add_argument("--instances", type=int, default=None,
                    help="instances of the batch (default: the workload's; smaller only for profiling captures)")
    ap.add_argument("--sweep", action="store_true",
                    help="time same-size batches on the M = N = K diagonal (prints its own JSON line)")
    ap.add_argument("--sweep-paths", default="ffma,3xbf16", type=lambda v: [x for x in v.split(",") if x],
                    help="FP32 paths of --sweep (name, name@stage, name@stream, name@warp)")
    ap.add_argument("--pack-ablation", action="store_true",
                    help="time the pack step against the no-pack path by size (prints its own JSON line)")
    ap.add_argument("--split", default="replicate", choices=["replicate", "shard"],
                    help="N>1 only: every rank runs the whole batch (replicate, weak scaling; the default) or "
                         "its contiguous cost-balanced shard of one batch (shard, strong scaling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plan with the built-in cost model instead of tuning each path first")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.pack_ablation:
        return run_pack_ablation(args)
    if args.sweep:
        return run_sweep(args)

    import torch
    import torch.distributed as dist

    rank, local_rank, world = env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    from paper_2208_09822_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2208_09822_gb300 import iaat
    from paper_2208_09822_gb300 import workloads as W

    # the autotuner (Sec. IV's install-time tuning, done at start-up here):
    # per-variant costs and the stage size of every timed path, measured on
    # this GPU before anything is timed; skipped when a tuning cache is given
    _, wl_desc, _, wl_dtype, wl_path, wl_tol = WORKLOADS[args.workload]
    if args.workload not in ("uneven", "uniform16"):
        # other batches: their type's CUDA-core path alone (the FP64 one on
        # the stage programs or, asked for, the warp-direct kernel)
        keep = lambda n: wl_dtype == 1 and ROUTE_BASE(n) == wl_path
        args.precision = args.precision if keep(args.precision) else wl_path
        args.compare = [n for n in args.compare if keep(n) and n != args.precision]

    tuned = "built-in cost model"
    if not args.no_autotune and not os.environ.get("IAAT_TUNE_CACHE") and wl_dtype in (0, 1):
        t0 = time.time()
        if wl_dtype == 0:
            names = [args.precision] + list(args.compare)
            precs = [PRECISIONS[n] for n in names] + [0 for n in names if n in ROUTE]
            for p in dict.fromkeys(precs):
                iaat.iaat_autotune(iaat.IAAT_F32, p, None)
        else:
            iaat.iaat_autotune(iaat.IAAT_F64, iaat.IAAT_PREC_DEFAULT, None)
        tuned = f"autotuned at start-up ({time.time() - t0:.1f} s, outside the timed region)"
    elif os.environ.get("IAAT_TUNE_CACHE"):
        tuned = "tuning cache " + os.environ["IAAT_TUNE_CACHE"]
    elif wl_dtype in (2, 3):
        tuned = "built-in cost model (the complex family is not autotuned)"

    batch = make_workload(args.workload, args.instances)
    # a batch that fits in L2 is timed over ROT copies of its pools, one per
    # launch in turn, so no launch finds its inputs in L2
    pool_bytes = batch.A.nbytes + batch.B.nbytes + batch.C.nbytes
    rot = 1 if pool_bytes > 129e6 else int(np.ceil(129e6 / pool_bytes)) + 1
    tile = (lambda x: x) if rot == 1 else (lambda x: np.tile(x, rot))
    tA_all = torch.from_numpy(tile(batch.A)).to(dev)
    tB_all = torch.from_numpy(tile(batch.B)).to(dev)
    tC_all = torch.from_numpy(tile(batch.C)).to(dev)
    tA, tB, tC = tA_all[:batch.A.size], tB_all[:batch.B.size], tC_all[:batch.C.size]
    C0 = tC.clone()
    to_descs = iaat.cdescs_for_pools if batch.is_complex else iaat.descs_for_pools
    descs_rot = [to_descs(batch, tA.data_ptr() + r * batch.A.nbytes, tB.data_ptr() + r * batch.B.nbytes,
                          tC.data_ptr() + r * batch.C.nbytes) for r in range(rot)]
    descs = descs_rot[0]
    stream = torch.cuda.Stream(device=dev)
    # the instances this rank runs: the whole batch, or its shard of it
    shard = args.split == "shard" and world > 1
    my = shard_ranges(batch, world)[rank] if shard else \
        {"i0": 0, "i1": batch.count, "flops": batch.flops(), "A": (0, batch.A.size), "B": (0, batch.B.size),
         "C": (0, batch.C.size)}
    r0, r1 = my["i0"], my["i1"]
    job_flops = batch.flops() if shard else batch.flops() * world   # every rank's instances together

    def make_plan(d, name):
        if wl_dtype == 0:
            rk, rm, rf = ROUTE.get(ROUTE_BASE(name), (0, 0, 0))
            return iaat.iaat_plan_create(d, iaat.IAAT_F32, PRECISIONS[name], route_k_below=rk, route_mnk_below=rm,
                                         route_kernel=rf, kernel=KERNEL.get(name, 0))
        if wl_dtype == 1:
            return iaat.iaat_plan_create(d, iaat.IAAT_F64, iaat.IAAT_PREC_DEFAULT, kernel=KERNEL.get(name, 0))
        return iaat.iaat_plan_create_complex(d, wl_dtype)

    # the DFMA-bound batches are held against the measured DFMA rate
    dfma_bound = wl_dtype in (1, 3)
    dfma_peak = iaat.iaat_fma_peak(iaat.IAAT_F64) if dfma_bound else None

    def route_split(d, name):
        """The two parts of a routed path's descriptors, by the planner's rule
        (K below route_k_below or M*N*K below route_mnk_below, alpha = 0
        counting as K = 0): (tensor-core part, CUDA-core part)."""
        rk, rm, _ = ROUTE[ROUTE_BASE(name)]
        keff = np.where(d["alpha"] == 0.0, 0, d["K"]).astype(np.int64)
        small = (keff < rk) | (d["M"].astype(np.int64) * d["N"] * keff < rm)
        return d[~small], d[small]

    def make_part(d, name, part):
        """Plan of one part of a routed path, alone (what that part's launch
        inside the routed plan runs)."""
        big, small = route_split(d, name)
        if part == 0:
            return iaat.iaat_plan_create(big, iaat.IAAT_F32, PRECISIONS[name], kernel=KERNEL.get(name, 0))
        return iaat.iaat_plan_create(small, iaat.IAAT_F32, iaat.IAAT_PREC_DEFAULT, kernel=ROUTE[ROUTE_BASE(name)][2])

    def time_path(name, part=None):
        """First launch (kept for the error check), then a CUDA graph of one
        launch per pool copy (one launch when the pools exceed L2) replayed
        between events on the launch stream, `steps` launches in all.  With
        `part` (0 tensor-core, 1 CUDA-core), one part of a routed path alone."""
        plans = [make_plan(d[r0:r1], name) if part is None else make_part(d[r0:r1], name, part) for d in descs_rot]
        plan = plans[0]
        info = iaat.iaat_plan_info(plan)
        tC.copy_(C0)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            iaat.iaat_gemm_grouped(plan, stream)
        iaat.iaat_plan_check(plan, stream)
        first = tC.cpu().numpy() if rank == 0 else None
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for p in plans:
                iaat.iaat_gemm_grouped(p, stream)
        replays = max(1, args.steps // rot)
        with torch.cuda.stream(stream):
            for _ in range(max(1, -(-args.warmup // rot))):
                g.replay()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):   # replay() launches on the current stream
            e0.record(stream)
            for _ in range(replays):
                g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = e0.elapsed_time(e1) / (replays * rot)
        for p in plans:
            iaat.iaat_plan_check(p, stream)
        for p in plans[1:]:
            p.destroy()
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return plan, info, ms, first

    # the compared paths first, then the headline path with the clock sampler
    others = [p for p in args.compare if p != args.precision]
    results = {}
    for name in others:
        plan_o, info_o, ms_o, first_o = time_path(name)
        results[name] = (info_o, ms_o, first_o)
        plan_o.destroy()
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.25)
    plan, info, ms, first_result = time_path(args.precision)
    clocks = sampler.stop()
    results[args.precision] = (info, ms, first_result)
    # a routed path's two launches, each timed alone: the roofline below is
    # the dominant one's (the path's own is kept beside it)
    parts = []
    if wl_dtype == 0 and ROUTE_BASE(args.precision) in ROUTE:
        for part, kname in ((0, "tensor-core part"), (1, "CUDA-core part")):
            plan_p, info_p, ms_p, _ = time_path(args.precision, part)
            parts.append({"part": kname, "kernel_family": info_p.get("kernel_family"), "ms": ms_p,
                          "instances": info_p["instances"], "algorithmic_bytes": info_p["algorithmic_bytes"]})
            plan_p.destroy()

    flops = info["flops"]
    value = job_flops / (ms * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    abytes = info["algorithmic_bytes"]
    achieved = abytes / (ms * 1e-3) / 1e9
    roof_gflops = abytes and flops / abytes * NOMINAL_HBM_GBS

    # end to end through the C ABI from pinned host buffers.  Serial: every
    # step copies the pools in, launches the plan, copies C out, one after the
    # other.  Pipelined (the reported number): the batch is cut into
    # contiguous instance ranges, one plan each, and on three streams the
    # copy-in of range c+1, the launch of range c and the copy-out of range c-1
    # overlap; a range is copied in again only after its previous copy-out.
    from paper_2208_09822_gb300.shard import instance_cost, shard_bounds
    hA = torch.from_numpy(batch.A).pin_memory()
    hB = torch.from_numpy(batch.B).pin_memory()
    hC = torch.from_numpy(batch.C).pin_memory()
    hOut = torch.empty_like(hC).pin_memory()
    (a0, a1), (b0_, b1_), (c0, c1) = my["A"], my["B"], my["C"]
    h2d = ((a1 - a0) * hA.element_size() + (b1_ - b0_) * hB.element_size() + (c1 - c0) * hC.element_size())
    d2h = (c1 - c0) * hOut.element_size()
    args.e2e_steps = max(1, args.e2e_steps)

    def copy_in_out(pl):
        tA[a0:a1].copy_(hA[a0:a1], non_blocking=True)
        tB[b0_:b1_].copy_(hB[b0_:b1_], non_blocking=True)
        tC[c0:c1].copy_(hC[c0:c1], non_blocking=True)
        iaat.iaat_gemm_grouped(pl, stream)
        hOut[c0:c1].copy_(tC[c0:c1], non_blocking=True)

    def e2e_serial():
        with torch.cuda.stream(stream):
            copy_in_out(plan)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(args.e2e_steps):
                copy_in_out(plan)
        f1.record(stream)
        torch.cuda.synchronize()
        return f0.elapsed_time(f1) / args.e2e_steps

    def e2e_pipelined(nchunks):
        n = batch.count
        cost = instance_cost(batch.M[r0:r1], batch.N[r0:r1], batch.K[r0:r1], batch.beta[r0:r1] != 0)
        ranges = [(r0 + b0, r0 + b1) for b0, b1 in shard_bounds(cost, nchunks) if b1 > b0]
        parts = []
        for b0, b1 in ranges:
            span = lambda off, pool: (int(off[b0]), int(off[b1]) if b1 < n else pool.size)
            parts.append((make_plan(descs[b0:b1], args.precision),
                          span(batch.offA, batch.A), span(batch.offB, batch.B), span(batch.offC, batch.C)))
        s_in = torch.cuda.Stream(device=dev)
        s_out = torch.cuda.Stream(device=dev)
        ev_in = [torch.cuda.Event() for _ in parts]
        ev_cmp = [torch.cuda.Event() for _ in parts]
        ev_out = [torch.cuda.Event() for _ in parts]

        def step(first):
            for c, (pl, ra, rb, rc) in enumerate(parts):
                if not first:
                    s_in.wait_event(ev_out[c])
                with torch.cuda.stream(s_in):
                    tA[ra[0]:ra[1]].copy_(hA[ra[0]:ra[1]], non_blocking=True)
                    tB[rb[0]:rb[1]].copy_(hB[rb[0]:rb[1]], non_blocking=True)
                    tC[rc[0]:rc[1]].copy_(hC[rc[0]:rc[1]], non_blocking=True)
                    ev_in[c].record(s_in)
                stream.wait_event(ev_in[c])
                iaat.iaat_gemm_grouped(pl, stream)
                ev_cmp[c].record(stream)
                s_out.wait_event(ev_cmp[c])
                with torch.cuda.stream(s_out):
                    hOut[rc[0]:rc[1]].copy_(tC[rc[0]:rc[1]], non_blocking=True)
                    ev_out[c].record(s_out)

        step(True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(s_in)
        stream.wait_event(f0)
        s_out.wait_event(f0)
        for _ in range(args.e2e_steps):
            step(False)
        s_out.wait_stream(s_in)
        s_out.wait_stream(stream)
        f1.record(s_out)
        torch.cuda.synchronize()
        for pl, *_ in parts:
            iaat.iaat_plan_check(pl, stream)
            pl.destroy()
        return f0.elapsed_time(f1) / args.e2e_steps, len(parts)

    e2e_serial_ms = e2e_serial()
    iaat.iaat_plan_check(plan, stream)
    e2e_ms, e2e_parts = e2e_pipelined(args.e2e_chunks)
    # the pipelined result must equal the one-plan result (same inputs, same
    # plans per instance); a mismatch withholds the end-to-end number
    e2e_ok = True
    if rank == 0 and not np.array_equal(hOut.numpy()[c0:c1].view(np.uint8), first_result[c0:c1].view(np.uint8)):
        e2e_ok = False
        print("error: pipelined end-to-end result differs from the single launch", file=sys.stderr)
    iaat.iaat_plan_check(plan, stream)
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = job_flops / (e2e_ms * 1e-3) / 1e9

    if rank == 0:
        cpu, errs = None, {}
        if world == 1 and not args.no_cpu_baseline:
            cpu, errs = cpu_baseline_leg(batch, {k: v[2] for k, v in results.items()}, 10.0, wl_tol)
        # a profile counts only for the kernel family this plan runs (the
        # autotuner may pick another one for a default path)
        traffic = profile_traffic(args.precision, args.workload, batch.count, info.get("kernel_family"))
        paths = {}
        for name, (inf, ms_p, _) in results.items():
            paths[name] = {"value": job_flops / (ms_p * 1e-3) / 1e9, "unit": "GFLOP/s",
                           "ms_per_step": ms_p, "launches_per_step": inf["kernels"],
                           "roofline_frac": inf["algorithmic_bytes"] / (ms_p * 1e-3) / 1e9 / peaks["hbm_gbs"],
                           "error": errs.get(name)}
        if dfma_bound:
            roofline = {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": dfma_peak / 1e3,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e9 / dfma_peak, "traffic": traffic,
                        "peak_kind": "measured DFMA rate (iaat_fma_peak, this GPU, at start-up)",
                        "algorithmic_bytes_per_launch": abytes,
                        "hbm_frac": achieved / peaks["hbm_gbs"]}
        elif parts:
            for pt in parts:
                pt["achieved_gbs"] = pt["algorithmic_bytes"] / (pt["ms"] * 1e-3) / 1e9
                pt["frac"] = pt["achieved_gbs"] / peaks["hbm_gbs"]
            dom = max(parts, key=lambda pt: pt["ms"])
            roofline = {"bound": "hbm", "achieved": dom["achieved_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": dom["frac"], "traffic": traffic,
                        "peak_kind": f"{peak_kind} copy bandwidth",
                        "kernel": f"{dom['part']} of the routed plan, timed alone",
                        "algorithmic_bytes_per_launch": dom["algorithmic_bytes"],
                        "path_achieved": achieved, "path_frac": achieved / peaks["hbm_gbs"],
                        "path_algorithmic_bytes_per_step": abytes, "parts": parts,
                        "roofline_gflops_at_8TBs": roof_gflops,
                        "frac_of_8TBs_roofline": value / world / roof_gflops if roof_gflops else None}
        else:
            roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                        "peak_kind": f"{peak_kind} copy bandwidth",
                        "algorithmic_bytes_per_launch": abytes,
                        "roofline_gflops_at_8TBs": roof_gflops,
                        "frac_of_8TBs_roofline": value / world / roof_gflops if roof_gflops else None}
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": max(1, args.steps // rot) * rot,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if shard else "weak",
            "vs_baseline": None, "dtype": DTYPE_NAMES[wl_dtype], "data": "synthetic",
            "config": {"workload": wl_desc.format(n=batch.count), "instances": batch.count,
                       "precision": args.precision,
                       "parallelism": (f"one batch cut into {world} contiguous cost-balanced shards, one per GPU"
                                       if shard else f"instances x{world} (one batch per GPU)"),
                       "l2": ("inputs larger than L2 (pools %.2f GB > 129 MB); no flush" % (pool_bytes / 1e9))
                             if rot == 1 else ("pools %.0f MB fit L2: launches rotate over %d copies (%.0f MB); "
                                               "no flush" % (pool_bytes / 1e6, rot, rot * pool_bytes / 1e6)),
                       "tasks": info["tasks"], "groups": info["groups"], "blocks": info["blocks"],
                       "grid": info["grid"], "tuning": tuned,
                       "kernel_family": {1: "stage programs", 2: "stream", 3: "warp-tile", 4: "warp-direct"}.get(
                           info.get("kernel_family"), "unknown") + (
                           " + warp-direct (routed part)" if ROUTE.get(ROUTE_BASE(args.precision), (0, 0, 0))[2] == 4
                           else "")},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value if e2e_ok else None, "unit": "GFLOP/s", "ok": e2e_ok,
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                    "pipelined_ranges": e2e_parts,
                    "serial_value": flops * world / (e2e_serial_ms * 1e-3) / 1e9},
            "paths": paths,
            "error": errs.get(args.precision),
            "gpu_launches": max(1, args.steps // rot) * rot * info["kernels"],
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0 if e2e_ok else 1


if __name__ == "__main__":
    sys.exit(main())
