#!/usr/bin/env python3
"""Benchmark of the dense -> symmetric band reduction (sy2sb) on one GB300.

Workload (the configuration the headline metric is quoted on): symmetric A of order
n = 8192 with a known spectrum, A = Q diag(lam) Q^T (Q from the QR factorisation of a
Gaussian matrix, lam log-uniform in [1e-6, 1] with random signs; seeds 0 and 1), reduced
to bandwidth w = 64 with panel width b = 64 and look-ahead.  One step = one complete
reduction of a fresh copy of A (the matrix is restored from a resident copy between steps,
outside the timed calls).  A is 512 MB, larger than the 129 MB L2, so no L2 flush is
needed between steps.

Metric: TFLOP/s with the nominal 4n^3/3 flop count of the method (Section 2.1).

The JSON line adds
  roofline      the dominant kernel class, timed live with CUDA events on its stream
                during the timed steps, against the measured peak of its bound;
  cpu_baseline  the FP64 oracle (one reflector at a time) on the host cores, on a bounded
                sample: the first reflectors of the same matrix;
  e2e           the same metric through the C ABI with host buffers: pinned host A ->
                device, reduction, device -> host of A and tau, all inside the timing;
  fp64_path     the plain FP64 GPU path on the same matrix, with its backward error;
  clocks        nvidia-smi samples taken during the timed steps.

--impl reference times the oracle instead (the CPU reference arm), each step one bounded
sample of the same workload.
Under torchrun (N > 1 GPUs) every rank reduces its own copy of the matrix (the single-
matrix reduction does not shard: replicas), the value is the work of all ranks over the
slowest rank's time, and only rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HEADLINE_METRIC = "band-reduction TFLOP/s & speedup vs FP64 path at equal backward error; mats/s"


def nominal_flops(n: int) -> float:
    return 4.0 * n ** 3 / 3.0


def sample_flops(n: int, w: int, ncols: int) -> float:
    """Nominal flops of the first ncols reflectors: reflector c updates a trailing matrix
    of order j_c = n - w - c from both sides (4 j_c^2 flops; the sum over c is 4n^3/3)."""
    return sum(4.0 * (n - w - c) ** 2 for c in range(ncols))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_traffic(kernel_name: str):
    """DRAM bytes per launch from a committed ncu capture, when the kernel source it was
    taken on is unchanged (its SHA-256 is stored with the figure); otherwise None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(kernel_name)
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src):
        return None
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != d["sha256"]:
            return None
    return d["dram_bytes_per_unit"]


def run_cpu_baseline(A_host, n, w, target_s: float):
    """Times the oracle on the first reflectors of the workload (bounded sample)."""
    import oracle

    cores = oracle.set_threads(0)
    # calibrate on a short prefix, then size the sample to about target_s seconds
    ncols = 8
    t0 = time.perf_counter()
    oracle.sy2sb(A_host, w, ncols=ncols)
    dt = time.perf_counter() - t0
    per = dt / sample_flops(n, w, ncols)
    ncols2 = ncols
    while ncols2 < n - w - 1 and sample_flops(n, w, ncols2 * 2) * per < target_s:
        ncols2 *= 2
    t0 = time.perf_counter()
    oracle.sy2sb(A_host, w, ncols=ncols2)
    dt = time.perf_counter() - t0
    fl = sample_flops(n, w, ncols2)
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"first {ncols2} of {n - w} reflectors of the n={n} w={w} workload ({dt:.1f} s; "
                      f"nominal flops of those reflectors)"}


def reference_arm(args, n, w, b):
    """CPU reference arm: the FP64 oracle, each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import workloads

    A, _ = workloads.sym_known_spectrum(n, 0, 1)
    cores = oracle.set_threads(0)
    ncols = args.ref_cols
    fl = sample_flops(n, w, ncols)
    for _ in range(args.warmup):
        oracle.sy2sb(A, w, ncols=max(2, ncols // 8))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sy2sb(A, w, ncols=ncols)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = fl / (ms / 1e3) / 1e12
    line = {
        "impl": "reference", "metric": HEADLINE_METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"sy2sb n={n} w={w} b={b} known-spectrum FP64 (bounded sample: first {ncols} "
                               f"reflectors per step)", "n": n, "w": w, "b": b},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {ncols} of {n - w} reflectors per step"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--w", type=int, default=64)
    ap.add_argument("--b", type=int, default=64)
    ap.add_argument("--precision", default="bf16x6", choices=["fp64", "bf16x3", "bf16x6", "ozaki"])
    ap.add_argument("--lookahead", type=int, default=-1)
    ap.add_argument("--no-fp64-path", action="store_true", help="skip the FP64 comparison line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-cols", type=int, default=96, help="reflectors per reference-arm step")
    args = ap.parse_args()
    n, w, b = args.n, args.w, args.b

    if args.impl == "reference":
        return reference_arm(args, n, w, b)

    import numpy as np
    import torch

    import paper_1709_00302_gb300 as br
    import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    br.build()
    br.lib()

    A_host, lam = workloads.sym_known_spectrum(n, 0, 1)
    A0 = torch.from_numpy(A_host).to(dev)  # column-major (Fortran) strides are kept
    A = torch.empty_like(A0)
    stream = torch.cuda.current_stream(dev)

    def make_call(precision, lookahead):
        o = br.make_opts(b=b, lookahead=lookahead, precision=precision)
        tau = torch.zeros(n - w, dtype=torch.float64, device=dev)
        work = torch.empty(br.bandred_sy2sb_workspace(n, w, o), dtype=torch.uint8, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)

        def call(M):
            rc = br.bandred_sy2sb_ex(M, w, tau, o, work, status, stream)
            if rc != 0:
                raise br.BandredError(rc, "bandred_sy2sb_ex")
        return call, tau, status

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed_steps(call, steps, warmup, profile=False):
        for _ in range(warmup):
            A.copy_(A0)
            call(A)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        l0 = br.bandred_launch_count()
        if profile:
            br.bandred_profile_begin()
        sampler = ClockSampler(local)
        sampler.start()
        for e0, e1 in ev:
            A.copy_(A0)
            e0.record(stream)
            call(A)
            e1.record(stream)
        barrier()
        clocks = sampler.stop()
        stats = br.bandred_profile_end() if profile else []
        launches = br.bandred_launch_count() - l0
        ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        return ms, stats, launches, clocks

    # ---- headline: the configured precision with look-ahead
    call, tau, status = make_call(args.precision, args.lookahead)
    ms, stats, launches, clocks = timed_steps(call, args.steps, args.warmup, profile=True)
    st = int(status.item())
    if st != 0:
        raise br.BandredError(st, "device status")
    my_ms = max(ms)
    ms_step = sum(ms) / len(ms)
    tot = torch.tensor([ms_step], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    ms_step_max = float(tot.item())
    value = world * nominal_flops(n) / (ms_step_max / 1e3) / 1e12

    # backward error of the headline result, estimated with Gaussian probes (test helper)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from checks import sym_probe_backward

    Aout = A.cpu().numpy()
    bwd = sym_probe_backward(A_host, Aout, tau.cpu().numpy(), w, probes=4)

    # ---- roofline of the dominant kernel class (live CUDA-event timing above)
    peaks, peak_src = load_peaks()
    dom = max(stats, key=lambda s: s["ms"]) if stats else None
    roof = None
    if dom is not None:
        per_launch_ms = dom["ms"] / dom["launches"]
        # The panel (FP64 reflectors) and the whole FP64 path are bound by the FP64 pipe;
        # the split-precision trailing updates stream A2 through HBM.
        alu = args.precision == "fp64" or dom["name"] in ("panel_qr_f64", "gemm")
        if alu:
            achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
            peak = 1.25
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "kernel": dom["name"], "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s; 1.20 measured "
                                                          "with an FMA loop)"}
        else:
            achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
            peak = peaks["hbm_gbs"]
            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "kernel": dom["name"], "peak_source": f"hbm_gbs ({peak_src})"}
        traffic = kernel_traffic(dom["name"])
        roof["traffic"] = None if traffic is None else traffic * dom["bytes"] / dom["launches"]
        roof["launches"] = dom["launches"]
        roof["avg_launch_ms"] = per_launch_ms
        roof["algorithmic_per_launch"] = (dom["flops"] if alu else dom["bytes"]) / dom["launches"]
        roof["kernels"] = {s["name"]: {"launches": s["launches"], "ms": s["ms"]} for s in stats}

    # ---- e2e through the C ABI with host buffers
    A_pin = torch.from_numpy(A_host).pin_memory()
    A_back = torch.empty_like(A_pin).pin_memory()
    tau_back = torch.empty(n - w, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for it in range(max(2, min(args.steps, 3)) + 1):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        A.copy_(A_pin, non_blocking=True)
        call(A)
        A_back.copy_(A, non_blocking=True)
        tau_back.copy_(tau, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if it > 0:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": nominal_flops(n) / (e2e_step / 1e3) / 1e12 * world, "unit": "TFLOP/s",
           "h2d_bytes_per_step": A_pin.numel() * 8, "d2h_bytes_per_step": A_back.numel() * 8 + tau_back.numel() * 8,
           "ms_per_step": e2e_step}

    # ---- plain FP64 GPU path on the same matrix (comparison line)
    fp64 = None
    if args.precision != "fp64" and not args.no_fp64_path:
        call64, tau64, _ = make_call("fp64", args.lookahead)
        ms64, _, _, _ = timed_steps(call64, 1, 1)
        b64 = sym_probe_backward(A_host, A.cpu().numpy(), tau64.cpu().numpy(), w, probes=4)
        fp64 = {"ms_per_step": ms64[0], "value": nominal_flops(n) / (ms64[0] / 1e3) / 1e12,
                "backward_error": b64, "speedup_of_headline": ms64[0] / ms_step}

    # ---- CPU baseline: the oracle on the host cores, bounded sample
    cpu = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(A_host, n, w, args.cpu_seconds)

    if rank == 0:
        dtype = {"fp64": "f64", "bf16x3": "bf16x3->f64", "bf16x6": "bf16x6->f64", "ozaki": "ozaki-bf16->f64"}
        line = {
            "metric": HEADLINE_METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype[args.precision], "data": "synthetic",
            "config": {"workload": f"sy2sb n={n} w={w} b={b} known-spectrum (lam log-uniform [1e-6,1], random "
                                   f"signs) precision={args.precision} lookahead={args.lookahead}",
                       "n": n, "w": w, "b": b, "precision": args.precision, "lookahead": args.lookahead,
                       "l2": "inputs (512 MB) larger than L2; matrix restored from a resident copy between steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "backward_error": bwd,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "fp64_path": fp64,
            "gpu_launches": launches,
            "clocks": clocks,
            "step_ms": ms,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
