#!/usr/bin/env python3
"""Benchmark of the dense -> symmetric band reduction (sy2sb) on one GB300.

Workload (the configuration the headline metric is quoted on): symmetric A of order
n = 8192 with a known spectrum, A = Q diag(lam) Q^T (Q from the QR factorisation of a
Gaussian matrix, lam log-uniform in [1e-6, 1] with random signs; seeds 0 and 1), reduced
to bandwidth w = 64 with panel width b = 64 and look-ahead.  One step = one complete
reduction of a fresh copy of A (the matrix is restored from a resident copy between steps,
outside the timed calls).  A is 512 MB, larger than the 129 MB L2, so no L2 flush is
needed between steps.

Metric: TFLOP/s with the nominal 4n^3/3 flop count of the method (Section 2.1), for the
precision that matches the FP64 path's backward error: the Ozaki scheme (FP64-accurate
products on the BF16 tensor cores).  Its speedup over the plain FP64 GPU path at equal
backward error is the metric's second part; mats/s (the batched workload) its third.

The JSON line adds
  roofline      the dominant kernel class, timed live with CUDA events on its stream
                during the timed steps, against the measured peak of its bound; the FP64
                rate of this GPU measured in the same run; the FP64 and split-precision
                rooflines of the step and its HBM fraction (12 sum j^2 bytes);
  cpu_baseline  the FP64 oracle (one reflector at a time) on the host cores, on a bounded
                sample: the first reflectors of the same matrix;
  e2e           the same metric through the C ABI with host buffers: pinned host A ->
                device, reduction, device -> host of A and tau, all inside the timing;
  fp64_path     the plain FP64 GPU path on the same matrix (several steps), with its
                backward error, and speedup_vs_fp64_at_equal_backward_error;
  bf16x6_path   the FP32-class split path on the same matrix, with its (larger) error;
  ge2gb, batched  compact records of the other two workloads (few steps);
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


DTYPES = {"fp64": "f64", "bf16x3": "bf16x3->f64", "bf16x6": "bf16x6->f64", "ozaki": "ozaki-bf16->f64"}


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
    """nvidia-smi samples (every 100 ms) kept for the timed region only: the sampler starts
    before the warm-up (so that nvidia-smi is already running when the timed steps begin),
    each line is stamped with its arrival time, and the statistics use the lines that
    arrived between mark_start() and one interval after mark_end()."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 100

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []  # (arrival time, line)
        self.thread = None
        self.t0 = None
        self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()
        if self.proc is not None:  # let the sample that covers the end of the region arrive
            time.sleep(1.5 * self.INTERVAL_MS / 1e3)

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
        lo = self.t0 if self.t0 is not None else float("-inf")
        hi = (self.t1 + self.INTERVAL_MS / 1e3) if self.t1 is not None else float("inf")
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if not lo <= t <= hi:
                continue
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


def ge2gb_sample_flops(m: int, n: int, w: int, ncols: int) -> float:
    """Nominal flops of the first ncols left/right reflector pairs: the left reflector of
    column c updates (m-c) x (n-c), the right one (m-c) x (n-c-w), 4 flops per entry each
    (the sum over all columns is 4(mn^2 - n^3/3) + O(w))."""
    return sum(4.0 * (m - c) * (n - c) + 4.0 * (m - c) * max(n - c - w, 0) for c in range(ncols))


def reference_arm(args, n, w, b):
    """CPU reference arm: the FP64 oracle, each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import workloads

    cores = oracle.set_threads(0)
    ncols = args.ref_cols
    wl = args.workload
    unit = "TFLOP/s"
    if wl == "batched":
        sym, gen = workloads.batched_mix(args.batch_sym, args.batch_gen, seed=0)
        k = max(1, ncols // 16)
        mats = [("sym", i, sym[i]) for i in range(k)] + [("gen", i, gen[i]) for i in range(k)]
        inputs = [workloads.batched_matrix(kind, i, (sh[0],) if kind == "sym" else sh[:2]) for kind, i, sh in mats]

        def step():
            for (kind, _, sh), M in zip(mats, inputs):
                if kind == "sym":
                    oracle.sy2sb(M, sh[1])
                else:
                    oracle.ge2gb(M, sh[2])
        units, unit = len(mats), "mats/s"
        desc = f"batched: the first {k} symmetric and {k} general matrices of the 1000 + 1000 mix per step"
        sample = f"{len(mats)} whole matrices per step"
        dtype_cfg = {"count": len(mats)}
    elif wl == "ge2gb":
        A = workloads.gen_gaussian(n, n, 0)

        def step():
            oracle.ge2gb(A, w, ncols=ncols)
        units = ge2gb_sample_flops(n, n, w, ncols)
        desc = (f"ge2gb m=n={n} w={w} b={b} N(0,1) precision=fp64 "
                f"(FP64 oracle; bounded sample: first {ncols} columns per step)")
        sample = f"first {ncols} of {n} left/right reflector pairs per step"
        dtype_cfg = {"m": n, "n": n, "w": w, "b": b}
    else:
        if wl == "sy2sb_large":
            G = np.random.Generator(np.random.PCG64(0)).standard_normal((n, n))
            A = np.asfortranarray((G + G.T) * 0.5)
            del G
            base = f"sy2sb n={n} w={w} b={b} N(0,1) symmetrised (drawn on the host: same distribution)"
        else:
            A, _ = workloads.sym_known_spectrum(n, 0, 1)
            base = f"sy2sb n={n} w={w} b={b} known-spectrum (lam log-uniform [1e-6,1], random signs)"

        def step():
            oracle.sy2sb(A, w, ncols=ncols)
        units = sample_flops(n, w, ncols)
        desc = f"{base} precision=fp64 (FP64 oracle; bounded sample: first {ncols} reflectors per step)"
        sample = f"first {ncols} of {n - w} reflectors per step"
        dtype_cfg = {"n": n, "w": w, "b": b}
    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = units / (ms / 1e3) / (1e12 if unit == "TFLOP/s" else 1.0)
    line = {
        "impl": "reference", "metric": HEADLINE_METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict({"workload": desc}, **dtype_cfg),
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_fp64_peak(br, dev, stream):
    """FP64 rate of this GPU, measured in the run: the library's FMA probe (eight
    independent FMA chains per thread, two CTAs of 512 threads per SM), timed with CUDA
    events on `stream`; the median of five launches after one warm-up launch."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = 2 * sms, 512, 4096
    sink = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    flops = 16.0 * blocks * threads * iters
    rates = []
    for it in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = br.bandred_fp64_probe(blocks, threads, iters, sink, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rc != 0:
            raise br.BandredError(rc, "bandred_fp64_probe")
        if it:
            rates.append(flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return {"tflops": statistics.median(rates), "best_tflops": max(rates), "launches": len(rates),
            "flops_per_launch": flops,
            "how": f"bandred_fp64_probe: {blocks} CTAs x {threads} threads x 8 chains x {iters} FP64 FMAs, "
                   f"CUDA events, median of {len(rates)} launches"}


def roofline(stats, precision, fp64_peak):
    """Roofline of the dominant kernel class of a profiled run: its algorithmic flops or
    bytes over its CUDA-event time, against the bound's peak (the FP64 rate measured in
    this run for the FP64-bound classes, MEASURED_PEAKS.json's copy bandwidth for the
    classes that stream the trailing matrix)."""
    peaks, peak_src = load_peaks()
    dom = max(stats, key=lambda s: s["ms"]) if stats else None
    if dom is None:
        return None
    per_launch_ms = dom["ms"] / dom["launches"]
    # The panel (FP64 reflectors) and the whole FP64 path are bound by the FP64 pipe;
    # the split-precision trailing updates stream the trailing matrix through HBM.
    alu = precision == "fp64" or dom["name"] == "panel_qr_f64"
    if alu:
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        peak = fp64_peak["tflops"]
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "kernel": dom["name"], "peak_source": "FP64 rate measured in this run (" + fp64_peak["how"] + ")"}
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
    roof["kernels"] = {s["name"]: {"launches": s["launches"], "ms": s["ms"],
                                   "tflops": s["flops"] / (s["ms"] / 1e3) / 1e12 if s["ms"] > 0 else None,
                                   "gbs": s["bytes"] / (s["ms"] / 1e3) / 1e9 if s["ms"] > 0 else None}
                       for s in stats}
    return roof


# digit-pair (or slice-pair) products per FP64 product of each split precision
PRODUCTS = {"ozaki": 28, "bf16x6": 6, "bf16x3": 3}


def step_rooflines(n, w, b, fp64_peak, times):
    """The step-level rooflines of the sy2sb workload.  Per iteration k the trailing update
    reads lower(A2) (X1 = A2 W), then reads and writes it (the rank-2k update): 12 j_k^2
    bytes, with j_k = n - w - k, for 4 j_k^2 b flops: an intensity of b/3 flop/byte.  The
    FP64 roofline is min(P_fp64, BW b/3); a split precision with p products per FP64
    product has min(P_bf16_sustained / p, BW b/3).  `times` maps a precision to its
    measured ms per step."""
    peaks, src = load_peaks()
    bw = peaks["hbm_gbs"] * 1e9
    algo_bytes = sum(12.0 * (n - w - k) ** 2 for k in range(0, n - w - 1, b))
    inten = nominal_flops(n) / algo_bytes
    out = {"algorithmic_bytes_per_step": algo_bytes, "intensity_flop_per_byte": inten,
           "hbm_gbs_peak": peaks["hbm_gbs"], "bf16_tflops_sustained": peaks.get("bf16_tflops_sustained"),
           "peaks_source": src}
    mem_roof = bw * inten / 1e12
    for prec, ms in times.items():
        if ms is None:
            continue
        achieved = nominal_flops(n) / (ms / 1e3) / 1e12
        if prec == "fp64":
            roof = min(fp64_peak["tflops"], mem_roof)
            bound = "fp64 pipe" if fp64_peak["tflops"] < mem_roof else "hbm"
        else:
            p = PRODUCTS[prec]
            roof = min(peaks["bf16_tflops_sustained"] / p, mem_roof)
            bound = f"bf16 tensor / {p}" if peaks["bf16_tflops_sustained"] / p < mem_roof else "hbm"
        out[prec] = {"roofline_tflops": roof, "bound": bound, "achieved_tflops": achieved, "frac": achieved / roof,
                     "hbm_gbs": algo_bytes / (ms / 1e3) / 1e9,
                     "hbm_frac": algo_bytes / (ms / 1e3) / bw}
    return out


def setup_distributed():
    import torch

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
    return world, rank, local, dist, dev


def make_problem(args, br, dev, stream):
    """Workload -> dict with the device input A0 (restored before every step), the call,
    the nominal flops of one step and the backward-error check."""
    import numpy as np
    import torch

    import workloads

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from checks import gen_probe_backward, sym_probe_backward

    wl = args.workload
    if wl in ("sy2sb", "sy2sb_large"):
        n, w, b = args.n, args.w, args.b
        if wl == "sy2sb_large":
            # 8.6 GB: drawn on the device (torch Philox, seed 0), symmetrised there
            g = torch.Generator(device=dev)
            g.manual_seed(0)
            G = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
            A0 = ((G + G.t()) * 0.5).t().contiguous().t()
            del G
            A_host = lam_true = None
            desc = f"sy2sb n={n} w={w} b={b} N(0,1) symmetrised (drawn on the device)"
        else:
            A_host, lam_true = workloads.sym_known_spectrum(n, 0, 1)
            A0 = torch.from_numpy(A_host).to(dev)
            desc = (f"sy2sb n={n} w={w} b={b} known-spectrum (lam log-uniform [1e-6,1], random signs)")

        def make_call(precision, lookahead):
            o = br.make_opts(b=b, lookahead=lookahead, precision=precision)
            tau = torch.zeros(n - w, dtype=torch.float64, device=dev)
            work = torch.empty(br.bandred_sy2sb_workspace(n, w, o), dtype=torch.uint8, device=dev)
            status = torch.zeros(1, dtype=torch.int32, device=dev)

            def call(M):
                rc = br.bandred_sy2sb_ex(M, w, tau, o, work, status, stream)
                if rc != 0:
                    raise br.BandredError(rc, "bandred_sy2sb_ex")
            return call, (tau,), status

        def backward(A, outs):
            if A_host is None:
                return None
            return sym_probe_backward(A_host, A.cpu().numpy(), outs[0].cpu().numpy(), w, probes=4)

        return dict(A0=A0, make_call=make_call, flops=nominal_flops(n), backward=backward, desc=desc,
                    config={"n": n, "w": w, "b": b}, units=1, lam=lam_true)
    if wl == "ge2gb":
        m = n = args.n
        w, b = args.w, args.b
        A_host = workloads.gen_gaussian(m, n, 0)
        A0 = torch.from_numpy(A_host).to(dev)

        def make_call(precision, lookahead):
            o = br.make_opts(b=b, lookahead=lookahead, precision=precision)
            tq = torch.zeros(n, dtype=torch.float64, device=dev)
            tp = torch.zeros(max(n - w, 0), dtype=torch.float64, device=dev)
            work = torch.empty(br.bandred_ge2gb_workspace(m, n, w, o), dtype=torch.uint8, device=dev)
            status = torch.zeros(1, dtype=torch.int32, device=dev)

            def call(M):
                rc = br.bandred_ge2gb_ex(M, w, tq, tp, o, work, status, stream)
                if rc != 0:
                    raise br.BandredError(rc, "bandred_ge2gb_ex")
            return call, (tq, tp), status

        def backward(A, outs):
            return gen_probe_backward(A_host, A.cpu().numpy(), outs[0].cpu().numpy(), outs[1].cpu().numpy(), w,
                                      probes=4)

        return dict(A0=A0, make_call=make_call, flops=4.0 * (m * n * n - n ** 3 / 3.0), backward=backward,
                    desc=f"ge2gb m=n={n} w={w} b={b} N(0,1)", config={"m": m, "n": n, "w": w, "b": b}, units=1)
    raise ValueError(wl)


def bench_batched(args, br, dev, stream, world, rank, dist, compact=False):
    """1000 symmetric (n ~ U[64,1024]) and 1000 general (n ~ U[64,1024], m ~ U[n,2n])
    matrices per GPU, w in {16, 32}; every step restores the inputs and replays one
    captured CUDA graph holding both batched runs.  With N ranks the batch is N times as
    large and split between them by LPT on nominal flops (paper_1709_00302_gb300.shard):
    no data crosses ranks, only the step times (max) and the status words (sum)."""
    import torch

    import workloads

    sym_all, gen_all = workloads.batched_mix(world * args.batch_sym, world * args.batch_gen, seed=0)
    if world > 1:
        from paper_1709_00302_gb300 import shard

        si, gi = shard.batched_shard(sym_all, gen_all, world, rank)
        sym, gen = [sym_all[i] for i in si], [gen_all[i] for i in gi]
    else:
        sym, gen = sym_all, gen_all
    total_count = len(sym_all) + len(gen_all)
    # one flat device buffer per kind; matrices are column-major views into it
    tot_s = sum(n * n for n, _ in sym)
    tot_g = sum(m * n for m, n, _ in gen)
    g = torch.Generator(device=dev)
    g.manual_seed(rank)
    flat_s0 = torch.randn(tot_s, dtype=torch.float64, device=dev, generator=g)
    flat_g0 = torch.randn(tot_g, dtype=torch.float64, device=dev, generator=g)
    flat_s, flat_g = flat_s0.clone(), flat_g0.clone()
    offs = [0]
    for n, _ in sym:
        offs.append(offs[-1] + n * n)
    offg = [0]
    for m, n, _ in gen:
        offg.append(offg[-1] + m * n)
    As, off = [], 0
    for n, _ in sym:
        v = flat_s[off:off + n * n].view(n, n).t()  # column-major view
        As.append(v)
        off += n * n
    # symmetrise each symmetric matrix's lower triangle source: (G + G^T)/2
    for a in As:
        a.copy_((a + a.t()) * 0.5)
    flat_s0.copy_(flat_s)
    Gs, off = [], 0
    for m, n, _ in gen:
        Gs.append(flat_g[off:off + m * n].view(n, m).t())
        off += m * n
    opts = br.make_opts(b=args.batch_b, precision=args.precision, panel_ctas=args.panel_ctas)
    taus = [torch.zeros(max(n - w, 0), dtype=torch.float64, device=dev) for n, w in sym]
    tqs = [torch.zeros(n, dtype=torch.float64, device=dev) for _, n, _ in gen]
    tps = [torch.zeros(max(n - w, 0), dtype=torch.float64, device=dev) for _, n, w in gen]
    sb = br.SyBatch(As, [w for _, w in sym], taus, opts)
    gb = br.GeBatch(Gs, [w for _, _, w in gen], tqs, tps, opts)
    ws = torch.empty(max(sb.workspace(), 256), dtype=torch.uint8, device=dev)
    wg = torch.empty(max(gb.workspace(), 256), dtype=torch.uint8, device=dev)
    st = torch.zeros(2, dtype=torch.int32, device=dev)
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(cap):
        assert sb.plan(ws, cap) == 0, br.bandred_last_error()
        assert gb.plan(wg, cap) == 0, br.bandred_last_error()
        cap.synchronize()
        graph = torch.cuda.CUDAGraph()
        l0 = br.bandred_launch_count()
        with torch.cuda.graph(graph, stream=cap):
            flat_s.copy_(flat_s0)
            flat_g.copy_(flat_g0)
            assert sb.run(ws, st[0:1], cap) == 0
            assert gb.run(wg, st[1:2], cap) == 0
        launches_per_step = br.bandred_launch_count() - l0
    # replays run on the current stream: make it the stream the events are recorded on
    with torch.cuda.stream(cap):
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        sampler.mark_start()
        for e0, e1 in ev:
            e0.record(cap)
            graph.replay()
            e1.record(cap)
        torch.cuda.synchronize(dev)
        sampler.mark_end()
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    assert int(st.sum().item()) == 0, st
    # one profiled step outside the graph: per-kernel-class times for the roofline
    with torch.cuda.stream(cap):
        flat_s.copy_(flat_s0)
        flat_g.copy_(flat_g0)
        torch.cuda.synchronize(dev)
        br.bandred_profile_begin()
        assert sb.run(ws, st[0:1], cap) == 0
        assert gb.run(wg, st[1:2], cap) == 0
        stats = br.bandred_profile_end()
    roof = roofline(stats, args.precision, measure_fp64_peak(br, dev, cap))
    # end to end: pinned host inputs -> device, both batched runs, outputs -> host
    hs, hg = flat_s0.cpu().pin_memory(), flat_g0.cpu().pin_memory()
    bs, bg = torch.empty_like(hs).pin_memory(), torch.empty_like(hg).pin_memory()
    e2e_ms = []
    with torch.cuda.stream(cap):
        for it in range(3):
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cap)
            flat_s.copy_(hs, non_blocking=True)
            flat_g.copy_(hg, non_blocking=True)
            assert sb.run(ws, st[0:1], cap) == 0
            assert gb.run(wg, st[1:2], cap) == 0
            bs.copy_(flat_s, non_blocking=True)
            bg.copy_(flat_g, non_blocking=True)
            e1.record(cap)
            torch.cuda.synchronize(dev)
            if it > 0:
                e2e_ms.append(e0.elapsed_time(e1))
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    tau_bytes = sum(t.numel() * 8 for t in taus + tqs + tps)
    e2e = {"value": total_count / (e2e_step / 1e3), "unit": "mats/s",
           "h2d_bytes_per_step": (hs.numel() + hg.numel()) * 8,
           "d2h_bytes_per_step": (bs.numel() + bg.numel()) * 8, "ms_per_step": e2e_step,
           "note": f"the packed outputs (band + reflectors) are copied back; the {tau_bytes} bytes of tau "
                   f"vectors stay on the device"}
    del hs, hg, bs, bg
    cpu = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline and not compact:
        import oracle

        cores = oracle.set_threads(0)
        t0 = time.perf_counter()
        done = 0
        for q in range(min(len(sym), len(gen))):
            n_, w_ = sym[q]
            oracle.sy2sb(flat_s0[offs[q]:offs[q] + n_ * n_].view(n_, n_).t().cpu().numpy(), w_)
            m_, n2, w2 = gen[q]
            oracle.ge2gb(flat_g0[offg[q]:offg[q] + m_ * n2].view(n2, m_).t().cpu().numpy(), w2)
            done += 2
            if time.perf_counter() - t0 > args.cpu_seconds:
                break
        dt = time.perf_counter() - t0
        cpu = {"value": done / dt, "unit": "mats/s", "cores": cores, "kind": "oracle",
               "sample": f"the first {done // 2} symmetric and {done // 2} general shapes of the mix ({dt:.1f} s)"}
    ms_step = sum(ms) / len(ms)
    t = torch.tensor([ms_step], dtype=torch.float64, device=dev)
    bad = st.sum().to(torch.float64).reshape(1)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(bad, op=dist.ReduceOp.SUM)  # device status words of every rank
    assert float(bad.item()) == 0.0, "a rank reported a device-side failure"
    ms_max = float(t.item())
    count = total_count
    value = count / (ms_max / 1e3)
    flops = sum(nominal_flops(n) for n, _ in sym_all) + sum(4.0 * (m * n * n - n ** 3 / 3.0) for m, n, _ in gen_all)
    # accuracy of one matrix of each kind, checked against its input on the host
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from checks import gen_probe_backward, sym_probe_backward

    i_s = max(range(len(sym)), key=lambda q: sym[q][0])
    i_g = max(range(len(gen)), key=lambda q: gen[q][1])
    n_s, w_s = sym[i_s]
    A_in = flat_s0[offs[i_s]:offs[i_s] + n_s * n_s].view(n_s, n_s).t().cpu().numpy()
    bw_s = sym_probe_backward(A_in, As[i_s].cpu().numpy(), taus[i_s].cpu().numpy(), w_s, probes=4)
    m_g, n_g, w_g = gen[i_g]
    G_in = flat_g0[offg[i_g]:offg[i_g] + m_g * n_g].view(n_g, m_g).t().cpu().numpy()
    bw_g = gen_probe_backward(G_in, Gs[i_g].cpu().numpy(), tqs[i_g].cpu().numpy(), tps[i_g].cpu().numpy(), w_g,
                              probes=4)
    if rank == 0:
        line = {
            "metric": HEADLINE_METRIC, "value": value, "unit": "mats/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": f"batched: {len(sym_all)} sy2sb n~U[64,1024] + {len(gen_all)} ge2gb n~U[64,1024] "
                                   f"m~U[n,2n], w in {{16,32}}, N(0,1) drawn on the device, one CUDA graph "
                                   f"replay per step" + (f", split over {world} GPUs by LPT on nominal flops"
                                                         if world > 1 else ""),
                       "count": count, "precision": args.precision,
                       "parallelism": f"batch sharded over {world} ranks" if world > 1 else "single",
                       "b": args.batch_b, "panel_ctas": args.panel_ctas, "l2": "inputs restored from resident copies inside the graph"},
            "tflops_nominal": flops / (ms_max / 1e3) / 1e12,
            "backward_error": {"sy2sb_largest": bw_s, "ge2gb_largest": bw_g},
            "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks, "step_ms": ms,
        }
        return line
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="sy2sb",
                    choices=["sy2sb", "ge2gb", "sy2sb_large", "batched", "paper_sweep"],
                    help="sy2sb: n=8192 w=b=64 known spectrum (headline); ge2gb: 8192^2 w=64; "
                         "sy2sb_large: n=32768 w=b=128; batched: 1000 + 1000 uneven matrices")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--w", type=int, default=None)
    ap.add_argument("--b", type=int, default=None)
    ap.add_argument("--precision", default="ozaki", choices=["fp64", "bf16x3", "bf16x6", "ozaki"])
    ap.add_argument("--lookahead", type=int, default=-1)
    ap.add_argument("--batch-sym", type=int, default=1000)
    ap.add_argument("--batch-gen", type=int, default=1000)
    ap.add_argument("--batch-b", type=int, default=0)
    ap.add_argument("--panel-ctas", type=int, default=0, help="panel_ctas option (batched: CTAs per matrix panel)")
    ap.add_argument("--no-fp64-path", action="store_true", help="skip the FP64 comparison line")
    ap.add_argument("--no-ozaki-path", action="store_true", help="skip the Ozaki-scheme comparison line")
    ap.add_argument("--no-bf16x6-path", action="store_true", help="skip the bf16x6 comparison line")
    ap.add_argument("--no-extras", action="store_true", help="skip the compact ge2gb and batched records")
    ap.add_argument("--cmp-steps", type=int, default=3, help="timed steps of each comparison path")
    ap.add_argument("--sweep-n", default="2500,5000,7500,10000", help="paper_sweep: orders n")
    ap.add_argument("--sweep-w", default="32,64,128,256", help="paper_sweep: bandwidths w")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-cols", type=int, default=96, help="reflectors per reference-arm step")
    args = ap.parse_args()
    defaults = {"sy2sb": (8192, 64, 64), "ge2gb": (8192, 64, 64), "sy2sb_large": (32768, 128, 128),
                "paper_sweep": (0, 0, 0),
                "batched": (0, 0, 0)}[args.workload]
    args.n = args.n or defaults[0]
    args.w = args.w or defaults[1]
    args.b = args.b or defaults[2]
    n, w, b = args.n, args.w, args.b

    if args.impl == "reference":
        return reference_arm(args, n, w, b)

    import torch

    import paper_1709_00302_gb300 as br

    world, rank, local, dist, dev = setup_distributed()
    br.build()
    br.lib()
    stream = torch.cuda.current_stream(dev)
    if args.workload == "paper_sweep":
        line = paper_sweep(args, br, dev, stream) if rank == 0 else None
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0
    if args.workload == "batched":
        line = bench_batched(args, br, dev, stream, world, rank, dist)
        if line is not None:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    prob = make_problem(args, br, dev, stream)
    A0 = prob["A0"]
    A = torch.empty_like(A0)
    A.copy_(A0)
    make_call = prob["make_call"]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed_steps(call, steps, warmup, profile=False):
        sampler = ClockSampler(local)
        sampler.start()
        for _ in range(warmup):
            A.copy_(A0)
            call(A)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        l0 = br.bandred_launch_count()
        if profile:
            br.bandred_profile_begin()
        sampler.mark_start()
        for e0, e1 in ev:
            A.copy_(A0)
            e0.record(stream)
            call(A)
            e1.record(stream)
        barrier()
        sampler.mark_end()
        clocks = sampler.stop()
        stats = br.bandred_profile_end() if profile else []
        launches = br.bandred_launch_count() - l0
        ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        return ms, stats, launches, clocks

    # ---- FP64 rate of this GPU (the FP64 roofline's denominator), measured before the timing
    fp64_peak = measure_fp64_peak(br, dev, stream)

    # ---- headline: the configured precision with look-ahead
    call, outs, status = make_call(args.precision, args.lookahead)
    ms, stats, launches, clocks = timed_steps(call, args.steps, args.warmup, profile=True)
    st = int(status.item())
    if st != 0:
        raise br.BandredError(st, "device status")
    ms_step = sum(ms) / len(ms)
    tot = torch.tensor([ms_step], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    ms_step_max = float(tot.item())
    value = world * prob["flops"] / (ms_step_max / 1e3) / 1e12
    bwd = prob["backward"](A, outs)

    # ---- roofline of the dominant kernel class (live CUDA-event timing above)
    roof = roofline(stats, args.precision, fp64_peak)

    # ---- e2e through the C ABI with host buffers
    A_pin = A0.cpu().pin_memory()
    A_back = torch.empty_like(A_pin).pin_memory()
    outs_back = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
    e2e_ms = []
    for it in range(max(2, min(args.steps, 3)) + 1):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        A.copy_(A_pin, non_blocking=True)
        call(A)
        A_back.copy_(A, non_blocking=True)
        for t, tb in zip(outs, outs_back):
            tb.copy_(t, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if it > 0:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": prob["flops"] / (e2e_step / 1e3) / 1e12 * world, "unit": "TFLOP/s",
           "h2d_bytes_per_step": A_pin.numel() * 8,
           "d2h_bytes_per_step": A_back.numel() * 8 + sum(t.numel() * 8 for t in outs_back),
           "ms_per_step": e2e_step}
    del A_pin, A_back

    def comparison(precision):
        """Another precision on the same matrix: --cmp-steps timed steps after one warm-up,
        median and spread, and its backward error."""
        c, o, stc = make_call(precision, args.lookahead)
        msc, _, _, _ = timed_steps(c, max(1, args.cmp_steps), 1)
        if int(stc.item()) != 0:
            raise br.BandredError(int(stc.item()), f"device status ({precision})")
        med = statistics.median(msc)
        return {"precision": precision, "steps": len(msc), "ms_per_step": med, "ms_min": min(msc),
                "ms_max": max(msc), "value": prob["flops"] / (med / 1e3) / 1e12, "unit": "TFLOP/s",
                "backward_error": prob["backward"](A, o)}

    # ---- plain FP64 GPU path on the same matrix: the denominator of the speedup at equal
    # backward error
    fp64 = None
    if args.precision != "fp64" and not args.no_fp64_path:
        fp64 = comparison("fp64")
        fp64["speedup_of_headline"] = fp64["ms_per_step"] / statistics.median(ms)
    ozaki = None
    if args.precision != "ozaki" and not args.no_ozaki_path:
        ozaki = comparison("ozaki")
        if fp64 is not None:
            ozaki["speedup_vs_fp64_path"] = fp64["ms_per_step"] / ozaki["ms_per_step"]
    bf16 = None
    if args.precision != "bf16x6" and not args.no_bf16x6_path:
        bf16 = comparison("bf16x6")
        bf16["note"] = "FP32-class products (six bf16 slice products): backward error about 1e-6, not FP64's"
        if fp64 is not None:
            bf16["speedup_vs_fp64_path"] = fp64["ms_per_step"] / bf16["ms_per_step"]
    eq = None
    if fp64 is not None and args.precision == "ozaki":
        eq = {"value": fp64["ms_per_step"] / statistics.median(ms), "fp64_ms_per_step": fp64["ms_per_step"],
              "ozaki_ms_per_step": statistics.median(ms), "fp64_backward_error": fp64["backward_error"],
              "ozaki_backward_error": bwd,
              "note": "median step times of the two paths on the same matrix, both at FP64-class backward error"}

    # ---- step rooflines (FP64 and split) and the step's HBM fraction
    step_roof = None
    if args.workload == "sy2sb":
        times = {args.precision: statistics.median(ms)}
        for cmp_ in (fp64, ozaki, bf16):
            if cmp_ is not None:
                times[cmp_["precision"]] = cmp_["ms_per_step"]
        step_roof = step_rooflines(n, w, b, fp64_peak, times)
    if roof is not None:
        roof["fp64_peak_measured"] = fp64_peak
        roof["step"] = step_roof

    # ---- compact records of the other workloads (few steps), so that one run observes all
    extras = {}
    if args.workload == "sy2sb" and not args.no_extras and world == 1:
        del A
        torch.cuda.empty_cache()
        extras["eigenvalues"] = compact_eigen(args, br, dev, stream, prob)
        torch.cuda.empty_cache()
        extras["singular_values"] = compact_svd(args, br, dev, stream, prob)
        torch.cuda.empty_cache()
        extras["ge2gb"] = compact_ge2gb(args, br, dev, stream)
        torch.cuda.empty_cache()
        extras["batched"] = compact_batched(args, br, dev, stream, world, rank, dist)
        torch.cuda.empty_cache()

    # ---- CPU baseline: the oracle on the host cores, bounded sample
    cpu = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline and args.workload == "sy2sb":
        cpu = run_cpu_baseline(A0.cpu().numpy(), n, w, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": HEADLINE_METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": dict({"workload": f"{prob['desc']} precision={args.precision} lookahead={args.lookahead}",
                            "precision": args.precision, "lookahead": args.lookahead,
                            "l2": "inputs larger than L2; matrix restored from a resident copy between steps",
                            "parallelism": "replicas" if world > 1 else "single"}, **prob["config"]),
            "backward_error": bwd,
            "speedup_vs_fp64_at_equal_backward_error": eq,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "fp64_path": fp64,
            "ozaki_path": ozaki,
            "bf16x6_path": bf16,
            "gpu_launches": launches,
            "clocks": clocks,
            "step_ms": ms,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def paper_sweep(args, br, dev, stream):
    """The paper's experiment shape (Section 4.2): symmetric matrices with entries uniform in
    (0, 1), n up to 10000, w in {32 .. 256}, b swept in steps of 16 up to w, with and without
    look-ahead (the variant b and w allow), timed per configuration (median of 2 runs after
    one warm-up) in the precision of --precision.  Reports TFLOP/s (4n^3/3) per point and the
    best b per (n, w) with and without look-ahead."""
    import torch

    ns = [int(x) for x in args.sweep_n.split(",")]
    ws = [int(x) for x in args.sweep_w.split(",")]
    rows, best = [], {}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    clocks.mark_start()
    for n in ns:
        g = torch.Generator(device=dev)
        g.manual_seed(n)
        U = torch.rand((n, n), dtype=torch.float64, device=dev, generator=g)
        A0 = ((U + U.t()) * 0.5).t().contiguous().t()
        del U
        A = torch.empty_like(A0)
        for w in ws:
            for b in range(16, w + 1, 16):
                for la in (0, -1):
                    o = br.make_opts(b=b, lookahead=la, precision=args.precision)
                    tau = torch.zeros(max(n - w, 1), dtype=torch.float64, device=dev)
                    work = torch.empty(br.bandred_sy2sb_workspace(n, w, o), dtype=torch.uint8, device=dev)
                    st = torch.zeros(1, dtype=torch.int32, device=dev)
                    ms = []
                    for it in range(3):
                        A.copy_(A0)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        rc = br.bandred_sy2sb_ex(A, w, tau, o, work, st, stream)
                        e1.record(stream)
                        torch.cuda.synchronize(dev)
                        if rc != 0 or int(st.item()) != 0:
                            raise br.BandredError(rc or int(st.item()), f"paper_sweep n={n} w={w} b={b}")
                        if it:
                            ms.append(e0.elapsed_time(e1))
                    med = statistics.median(ms)
                    tf = nominal_flops(n) / (med / 1e3) / 1e12
                    rows.append([n, w, b, la, round(med, 3), round(tf, 3)])
                    key = f"n{n}/w{w}/la{'auto' if la else 'none'}"
                    if key not in best or tf > best[key][1]:
                        best[key] = (b, round(tf, 3))
        del A, A0
        torch.cuda.empty_cache()
    clocks.mark_end()
    return {"metric": HEADLINE_METRIC, "workload": "paper_sweep", "unit": "TFLOP/s", "precision": args.precision,
            "data": "synthetic uniform (0,1) symmetric, drawn on the device",
            "columns": ["n", "w", "b", "lookahead", "ms", "tflops"], "rows": rows,
            "best_b": {k: {"b": v[0], "tflops": v[1]} for k, v in best.items()}, "clocks": clocks.stop()}


def compact_eigen(args, br, dev, stream, prob):
    """The whole eigenvalue path on the headline's matrix (the paper's two-stage solver:
    band reduction, band -> tridiagonal, tridiagonal eigenvalues): sy2sb in the Ozaki
    precision, then bandred_sb2st and bandred_sterf, each timed with CUDA events over one
    run after one warm-up, with the largest eigenvalue error against the known spectrum."""
    import ctypes

    import numpy as np
    import torch

    n, w, b = args.n, args.w, args.b
    A0 = prob["A0"]
    A = torch.empty_like(A0)
    o = br.make_opts(b=b, lookahead=args.lookahead, precision="ozaki")
    tau = torch.zeros(n - w, dtype=torch.float64, device=dev)
    work = torch.empty(br.bandred_sy2sb_workspace(n, w, o), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    e = torch.zeros(max(n - 1, 1), dtype=torch.float64, device=dev)
    lam = torch.zeros(n, dtype=torch.float64, device=dev)
    w2 = torch.empty(max(br.lib().bandred_sb2st_workspace(n, w), 256), dtype=torch.uint8, device=dev)
    w3 = torch.empty(max(br.lib().bandred_sterf_workspace(n), 256), dtype=torch.uint8, device=dev)
    st2 = torch.zeros(1, dtype=torch.int32, device=dev)
    L = br.lib()
    P = ctypes.c_void_p
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(2):
        A.copy_(A0)
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        if br.bandred_sy2sb_ex(A, w, tau, o, work, st, stream) != 0:
            raise br.BandredError(-1, "bandred_sy2sb_ex")
        ev[1].record(stream)
        rc = L.bandred_sb2st(n, w, P(A.data_ptr()), A.stride(1), P(d.data_ptr()), P(e.data_ptr()), None,
                             P(w2.data_ptr()), w2.numel(), P(st2.data_ptr()), P(stream.cuda_stream))
        if rc != 0:
            raise br.BandredError(rc, "bandred_sb2st")
        ev[2].record(stream)
        rc = L.bandred_sterf(n, P(d.data_ptr()), P(e.data_ptr()), P(lam.data_ptr()), P(w3.data_ptr()), w3.numel(),
                             P(stream.cuda_stream))
        if rc != 0:
            raise br.BandredError(rc, "bandred_sterf")
        ev[3].record(stream)
        torch.cuda.synchronize(dev)
    if int(st.item()) != 0 or int(st2.item()) != 0:
        raise br.BandredError(int(st.item()) or int(st2.item()), "device status (eigenvalue path)")
    ms = [ev[q].elapsed_time(ev[q + 1]) for q in range(3)]
    out = {"workload": prob["desc"] + " precision=ozaki, then band -> tridiagonal and bisection",
           "sy2sb_ms": ms[0], "sb2st_ms": ms[1], "sterf_ms": ms[2], "total_ms": sum(ms)}
    if prob.get("lam") is not None:
        lt = np.sort(np.asarray(prob["lam"]))
        out["max_eig_error_rel"] = float(np.max(np.abs(lam.cpu().numpy() - lt)) / np.max(np.abs(lt)))
    del A
    return out


def compact_svd(args, br, dev, stream, prob):
    """The whole singular-value path on the headline's matrix (its singular values are
    the absolute values of its known eigenvalues): ge2gb in the Ozaki precision (the
    general reduction to upper band form), then bandred_gb2bd and bandred_bdsv, each timed
    with CUDA events over one run after one warm-up."""
    import ctypes

    import numpy as np
    import torch

    n, w, b = args.n, args.w, args.b
    A0 = prob["A0"]
    A = torch.empty_like(A0)
    o = br.make_opts(b=b, lookahead=args.lookahead, precision="ozaki")
    tauq = torch.zeros(n, dtype=torch.float64, device=dev)
    taup = torch.zeros(max(n - w, 1), dtype=torch.float64, device=dev)
    work = torch.empty(max(br.bandred_ge2gb_workspace(n, n, w, o), 256), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    e = torch.zeros(max(n - 1, 1), dtype=torch.float64, device=dev)
    sig = torch.zeros(n, dtype=torch.float64, device=dev)
    L = br.lib()
    w2 = torch.empty(max(L.bandred_gb2bd_workspace(n, w), 256), dtype=torch.uint8, device=dev)
    w3 = torch.empty(max(L.bandred_bdsv_workspace(n), 256), dtype=torch.uint8, device=dev)
    st2 = torch.zeros(1, dtype=torch.int32, device=dev)
    P = ctypes.c_void_p
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(2):
        A.copy_(A0)
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        if br.bandred_ge2gb_ex(A, w, tauq, taup, o, work, st, stream) != 0:
            raise br.BandredError(-1, "bandred_ge2gb_ex")
        ev[1].record(stream)
        rc = L.bandred_gb2bd(n, w, P(A.data_ptr()), A.stride(1), P(d.data_ptr()), P(e.data_ptr()), None,
                             P(w2.data_ptr()), w2.numel(), P(st2.data_ptr()), P(stream.cuda_stream))
        if rc != 0:
            raise br.BandredError(rc, "bandred_gb2bd")
        ev[2].record(stream)
        rc = L.bandred_bdsv(n, P(d.data_ptr()), P(e.data_ptr()), P(sig.data_ptr()), P(w3.data_ptr()), w3.numel(),
                            P(stream.cuda_stream))
        if rc != 0:
            raise br.BandredError(rc, "bandred_bdsv")
        ev[3].record(stream)
        torch.cuda.synchronize(dev)
    if int(st.item()) != 0 or int(st2.item()) != 0:
        raise br.BandredError(int(st.item()) or int(st2.item()), "device status (singular-value path)")
    ms = [ev[q].elapsed_time(ev[q + 1]) for q in range(3)]
    out = {"workload": prob["desc"].replace("sy2sb", "ge2gb") + " precision=ozaki, then band -> bidiagonal and "
           "trisection on the Golub-Kahan tridiagonal",
           "ge2gb_ms": ms[0], "gb2bd_ms": ms[1], "bdsv_ms": ms[2], "total_ms": sum(ms)}
    if prob.get("lam") is not None:
        st_ = np.sort(np.abs(np.asarray(prob["lam"])))[::-1]
        out["max_sv_error_rel"] = float(np.max(np.abs(sig.cpu().numpy() - st_)) / st_[0])
    del A
    return out


def compact_ge2gb(args, br, dev, stream):
    """ge2gb m = n = 8192, w = b = 64, N(0,1), Ozaki precision: 3 timed steps after one
    warm-up, with its probe backward error."""
    import torch

    a2 = argparse.Namespace(**vars(args))
    a2.workload, a2.n, a2.w, a2.b = "ge2gb", 8192, 64, 64
    prob = make_problem(a2, br, dev, stream)
    A0 = prob["A0"]
    A = torch.empty_like(A0)
    call, outs, st = prob["make_call"]("ozaki", args.lookahead)
    A.copy_(A0)
    call(A)
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(3):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call(A)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    if int(st.item()) != 0:
        raise br.BandredError(int(st.item()), "device status (ge2gb)")
    med = statistics.median(ms)
    out = {"workload": prob["desc"] + " precision=ozaki", "steps": len(ms), "ms_per_step": med,
           "value": prob["flops"] / (med / 1e3) / 1e12, "unit": "TFLOP/s (4(mn^2 - n^3/3))",
           "backward_error": prob["backward"](A, outs), "step_ms": ms}
    del A, A0
    return out


def compact_batched(args, br, dev, stream, world, rank, dist):
    """The batched workload (1000 + 1000 uneven matrices, bf16x6: the batched path has no
    FP64-class precision) with 2 timed graph replays after one warm-up."""
    a2 = argparse.Namespace(**vars(args))
    a2.workload, a2.precision, a2.steps, a2.warmup = "batched", "bf16x6", 2, 1
    line = bench_batched(a2, br, dev, stream, world, rank, dist, compact=True)
    if line is None:
        return None
    keep = ("value", "unit", "ms_per_step", "steps", "dtype", "tflops_nominal", "backward_error", "config")
    out = {k: line[k] for k in keep if k in line}
    out["e2e_mats_per_s"] = line["e2e"]["value"] if line.get("e2e") else None
    return out


if __name__ == "__main__":
    sys.exit(main())
