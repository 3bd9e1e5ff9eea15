#!/usr/bin/env python3
"""Benchmark: batched permanents of n = 20 matrices on one GB300 (or N replicas).

One step = one pass of the whole hot path over one batch: 4096 complex128
20x20 submatrices of a 400x400 Haar unitary (rows 0..19, random sorted
20-column subsets) and 4096 Bernoulli(0.5) 20x20 0/1 matrices, each batch
through perm_batch (Store-zechin, one CTA per matrix, persistent launch).

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (the deliberately plain double-double / exact Ryser of Eq. (4)) on a
bounded sample of the same workload.

Extra measurements (on by default, bounded): the plain one-matrix-per-launch
form on a sample, the single n = 32 complex matrix with both kernels, and the
serving loop under Poisson arrivals (p50/p99 latency).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 20
COUNT = 4096
METRIC = ("n=20 permanents/s (4096 complex128 by batched Store-zechin + 4096 0/1 exact "
          "by the integer default, Ryser, per step)")
UNIT = "permanents/s"
WORKLOAD = ("n=20 batched: 4096 complex128 submatrices of a seeded 400x400 Haar unitary "
            "(rows 0..19, uniform sorted 20-column subsets) + 4096 seeded Bernoulli(0.5) 20x20 0/1 matrices")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libperm", choices=["libperm", "reference"])
    ap.add_argument("--count", type=int, default=COUNT)
    ap.add_argument("--no-extras", action="store_true", help="skip plain / n=32 / serving measurements")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--case", default="bench", choices=["bench", "single"],
                    help="single: one matrix of order --n with --method (for profiling)")
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--method", default="sz", choices=["sz", "ryser"])
    ap.add_argument("--dtype", default="c128", choices=["c128", "u01", "i64"])
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default CTA size and chain width (profiling runs)")
    ap.add_argument("--int-method", default="auto", choices=["auto", "sz"],
                    help="method of the 0/1 half: auto (Ryser, the default for integers) or sz "
                         "(the integer Store-zechin kernel; for profiling it)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per n = 20 complex matrix of sz_batched_c128, from the ncu capture
# summarised in profiles/sz_batched_c128_n20.md (304 matrices: 29.766018 GB + 7.642920 GB).
# Valid only for the kernel source it was measured on; otherwise the bench reports null.
TRAFFIC_C128_PER_MATRIX = (29.766018e9 + 7.642920e9) / 304
TRAFFIC_SOURCE_SHA256 = "6bae25e5546f5c116f1a0761fe0cfad8f4beb31e333d40f41125b77b5e464648"


def traffic_per_launch(count: int):
    import hashlib
    src = os.path.join(ROOT, "paper_1802_02779_gb300", "csrc", "sz_kernels.cu")
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != TRAFFIC_SOURCE_SHA256:
            return None
    return TRAFFIC_C128_PER_MATRIX * count


# ---------------------------------------------------------------------------
# multi-GPU replicas: max-over-ranks time and the whole-job rate
# ---------------------------------------------------------------------------
def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Units all replicas processed divided by the slowest replica's time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------
# algorithmic work (per permanent) for the roofline
# ---------------------------------------------------------------------------
def sz_c128_flops(n: int) -> float:
    """FP64 flops the complex Store-zechin kernel executes per n x n permanent.

    Each term a[k-1][j] * T_{k-1}[S \\ j] of a level 2 <= k <= n-1 entry is three
    FMAs (6 flops, three-multiplication complex form); each such entry adds 3
    additions (Re = P1-P2, w = P3-2 P2, Im = w-Re).  Level 1 is a copy; the
    final level (n terms in double-double) is negligible and not counted."""
    from math import comb
    f = 0.0
    for k in range(2, n):
        f += comb(n, k) * (6.0 * k + 3.0)
    return f


def sz_c128_standard_flops(n: int) -> float:
    """The same work counted the classical way: the method's n(2^(n-1)-1) complex
    multiplications at 6 flops and (n-2)2^(n-1)+1 complex additions at 2 flops."""
    return 6.0 * n * (2 ** (n - 1) - 1) + 2.0 * ((n - 2) * 2 ** (n - 1) + 1)


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def cpu_oracle_rate(cmats, imats, seconds: float):
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    done_c = done_i = 0
    k = 0
    while time.perf_counter() - t0 < seconds and k < len(cmats):
        oracle.per_ryser(cmats[k])
        done_c += 1
        oracle.per_ryser(imats[k])
        done_i += 1
        k += 1
    dt = time.perf_counter() - t0
    return (done_c + done_i) / dt, cores, done_c, done_i, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1802_02779_gb300 import workloads as wl
    cm, im = wl.batched_n20(count=64)
    rates = []
    total = 0
    for _ in range(args.warmup):
        cpu_oracle_rate(cm[:1], im[:1], 1e9)
    per_step_s = max(1.0, args.cpu_seconds / max(1, args.steps))
    for s in range(args.steps):
        r, cores, dc, di, dt = cpu_oracle_rate(cm[s % 8 * 8:], im[s % 8 * 8:], per_step_s)
        rates.append(r)
        total += dc + di
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * 2 * COUNT / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "dd/exact-int",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{total} matrices of the workload (half complex, half 0/1), "
                                       f"~{per_step_s:.0f} s per step, double-double / exact Ryser Eq. (4) with OpenMP"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, rank, world):
    import torch
    from paper_1802_02779_gb300 import build, libperm as lp, workloads as wl
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    build.build()
    lp.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    count = args.count
    cm, im = wl.batched_n20(count=count)
    c_host = torch.from_numpy(np.ascontiguousarray(cm).reshape(-1)).pin_memory()
    i_host = torch.from_numpy(np.ascontiguousarray(im).reshape(-1)).pin_memory()
    c_dev = c_host.cuda()
    i_dev = i_host.cuda()
    sizes = [N] * count
    c_out = torch.empty(count, dtype=torch.complex128, device="cuda")
    i_out = torch.empty((count, 2), dtype=torch.int64, device="cuda")
    c_st = torch.empty(count, dtype=torch.int32, device="cuda")
    i_st = torch.empty(count, dtype=torch.int32, device="cuda")
    tune = 0 if args.no_autotune else lp.FLAG_AUTOTUNE
    pc = lp.Plan(N, "c128", max_batch=count, flags=tune)
    pi = lp.Plan(N, "u01", max_batch=count, flags=tune,
                 method=lp.METHOD_SZ if args.int_method == "sz" else lp.METHOD_AUTO)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        pc.batch(c_dev, sizes, c_out, c_st, stream)
        pi.batch(i_dev, sizes, i_out, i_st, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # correctness guard on the timed buffers: all statuses OK
    assert int(c_st.abs().sum()) == 0 and int(i_st.abs().sum()) == 0

    fp64_peak = lp.measure_fp64_peak(300.0) if rank == 0 else 0.0

    clocks = Clocks(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (256 MB write, untimed)
        e0, e1, e2 = ev[k]
        e0.record(stream)
        pc.batch(c_dev, sizes, c_out, c_st, stream)
        e1.record(stream)
        pi.batch(i_dev, sizes, i_out, i_st, stream)
        e2.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    c_ms = [a.elapsed_time(b) for a, b, c in ev]
    i_ms = [b.elapsed_time(c) for a, b, c in ev]
    total_ms = max_over_ranks(float(np.sum(step_ms)), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(2 * count, world, ms_per_step / 1000.0)

    # ---- e2e: host buffers through perm_batch_host, copies inside the timed region ----
    ch_np = np.ascontiguousarray(cm).reshape(-1)
    ih_np = np.ascontiguousarray(im).reshape(-1)
    ch_pin = torch.from_numpy(ch_np).pin_memory().numpy()
    ih_pin = torch.from_numpy(ih_np).pin_memory().numpy()
    co = torch.empty(count * 2, dtype=torch.float64).pin_memory().numpy()
    io = torch.empty(count * 2, dtype=torch.int64).pin_memory().numpy()
    for _ in range(2):
        pc.batch_host(ch_pin, sizes, co, None, stream)
        pi.batch_host(ih_pin, sizes, io, None, stream)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pc.batch_host(ch_pin, sizes, co, None, stream)
        pi.batch_host(ih_pin, sizes, io, None, stream)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, "cuda")
    e2e = {"value": whole_job_rate(2 * count, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(ch_np.nbytes + ih_np.nbytes), "d2h_bytes_per_step": int(count * 16 * 2)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    c_kernel_ms = float(np.mean(c_ms))
    # launches per step: the batched complex kernel, the layer launches (t + 1 of them) of its
    # last partial round when the batch is not a whole number of rounds, then the 0/1 half
    # (Ryser: width, Gray-code and finishing kernels; --int-method sz: one batched kernel)
    dc = pc.describe()
    tail = count % dc["batched_grid"] if count > dc["batched_grid"] else 0
    tail_m = dc["chain_width_layer_small"] if N <= dc["layer_small_nmax"] else dc["chain_width_single"]
    launches_per_step = 1 + ((N - tail_m + 1) if tail else 0) + (1 if args.int_method == "sz" else 3)
    # achieved: the method's own work per permanent (n(2^(n-1)-1) complex multiplications at
    # 6 flops, (n-2)2^(n-1)+1 complex additions at 2), the per-unit figure of the roofline
    flops = sz_c128_standard_flops(N) * count
    achieved = flops / (c_kernel_ms / 1000.0) / 1e12
    executed = sz_c128_flops(N) * count / (c_kernel_ms / 1000.0) / 1e12
    peak = fp64_peak / 1e12
    roofline = {"bound": "alu", "pipe": "fp64", "kernel": "sz_batched_c128",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "measured this run by perm_measure_fp64_peak (independent DFMA chains, all SMs)",
                "work_per_permanent_flops": sz_c128_standard_flops(N),
                "work_count": "the method's complex multiplications x 6 + complex additions x 2",
                "executed_flops_per_permanent": sz_c128_flops(N),
                "executed_tflops": executed, "executed_frac": executed / peak,
                "traffic": traffic_per_launch(count),
                "traffic_unit": "bytes per launch (ncu dram__bytes_read+write, scaled per matrix)"}

    extras = {}
    if not args.no_extras:
        extras = measure_extras(lp, torch, cm, im, stream, c_kernel_ms, count)

    # ---- CPU baseline: the oracle on a bounded sample ----
    r, cores, dc, di, dt = cpu_oracle_rate(cm[:64], im[:64], args.cpu_seconds)
    cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{dc} complex + {di} 0/1 matrices of the workload in {dt:.1f} s "
                     f"(double-double / exact Ryser Eq. (4), OpenMP)"}

    metric = METRIC if args.int_method != "sz" else METRIC.replace("by the integer default, Ryser",
                                                                   "by Store-zechin (--int-method sz)")
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "complex128": count, "zero_one": count,
                       "method": {"complex128": "Store-zechin, persistent batched launch (one CTA per matrix)",
                                  "zero_one": ("Store-zechin batched 0/1 kernel, register rows (--int-method sz)"
                                               if args.int_method == "sz" else
                                               "Ryser Gray-code kernel (PERM_METHOD_AUTO's method for integers): "
                                               "width kernel, one CTA per 2^16 Glynn codes, finishing kernel")},
                       "l2": "flushed between timed steps (256 MB write)",
                       "plans": {"complex128": pc.describe(), "zero_one": pi.describe()},
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "complex_perm_per_s": count / (c_kernel_ms / 1000.0),
            "zero_one_perm_per_s": count / (float(np.mean(i_ms)) / 1000.0),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": ck}
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def measure_extras(lp, torch, cm, im, stream, c_kernel_ms, count):
    out = {}
    # plain: one matrix per launch sequence (whole GPU per matrix), on a sample
    sample = 32
    c_dev = torch.from_numpy(np.ascontiguousarray(cm[:sample]).reshape(-1)).cuda()
    o = torch.empty(sample, dtype=torch.complex128, device="cuda")
    with lp.Plan(N, "c128", flags=lp.FLAG_PLAIN, max_batch=sample) as pp:
        few_m = pp.describe()["chain_width_layer_few_n20"]
        pp.batch(c_dev, [N] * sample, o, None, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pp.batch(c_dev, [N] * sample, o, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms = e0.elapsed_time(e1)
    out["plain_vs_batched"] = {
        "plain_complex_perm_per_s": sample / (plain_ms / 1000.0),
        "batched_complex_perm_per_s": count / (c_kernel_ms / 1000.0),
        "speedup": (count / c_kernel_ms) / (sample / plain_ms),
        "plain_sample": sample,
        "plain": f"one matrix at a time over the whole GPU (Store-zechin chains of 2^{few_m}, one dataflow "
                 "launch per matrix)"}
    # single n = 32 instance, both kernels
    from paper_1802_02779_gb300 import workloads as wl
    a32 = wl.single_n32()
    d32 = torch.from_numpy(a32.reshape(-1)).cuda()
    o32 = torch.empty(2, dtype=torch.complex128, device="cuda")
    res = {}
    for name, meth in (("store_zechin", lp.METHOD_SZ), ("ryser", lp.METHOD_RYSER)):
        with lp.Plan(32, "c128", method=meth, max_batch=1) as p32:
            p32.batch(d32, [32], o32[:1], None, stream)     # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p32.batch(d32, [32], o32[:1], None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            res[name + "_ms"] = e0.elapsed_time(e1)
            res[name + "_value"] = [float(o32[0].real), float(o32[0].imag)]
    res["sz_work_tflops"] = sz_c128_standard_flops(32) / (res["store_zechin_ms"] / 1000.0) / 1e12
    out["n32"] = res
    out["n34"] = measure_n34(lp, torch, stream)
    out["n35"] = measure_n34(lp, torch, stream, n=35, budget_gb=200)
    out["integer_methods"] = measure_integer_methods(lp, torch, im, stream, count)
    out["wide"] = measure_wide(lp, torch, stream)
    out["five_boson"] = measure_five_boson(lp, torch, stream)
    out["uneven"] = measure_uneven(lp, torch, stream)
    out["serving_n20"] = measure_serving_n20(lp)
    out["serving"] = measure_serving(lp)
    return out


def _event_ms(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_n34(lp, torch, stream, n=34, budget_gb=150):
    """The largest Store-zechin orders, n = 34 and 35 complex (compact chain tables of 16 B
    per entry in HBM: 92 and 185 GB), one seeded matrix of the single-instance kind, against
    Ryser on the same matrix."""
    g = np.random.default_rng(18000 + n)
    a = ((g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2.0) / n).astype(np.complex128)
    d = torch.from_numpy(a.reshape(-1)).cuda()
    o = torch.empty(1, dtype=torch.complex128, device="cuda")
    res = {"n": n}
    for name, meth, budget in (("store_zechin", lp.METHOD_SZ, budget_gb << 30), ("ryser", lp.METHOD_RYSER, 0)):
        with lp.Plan(n, "c128", method=meth, max_batch=1, mem_budget_bytes=budget) as p:
            if name == "store_zechin":
                res["workspace_gb"] = p.workspace_bytes() / 1e9
            res[name + "_ms"] = _event_ms(torch, stream, lambda: p.batch(d, [n], o, None, stream))
            res[name + "_value"] = [float(o[0].real), float(o[0].imag)]
    res["sz_work_tflops"] = sz_c128_standard_flops(n) / (res["store_zechin_ms"] / 1000.0) / 1e12
    return res


def measure_integer_methods(lp, torch, im, stream, count):
    """The 4096 0/1 matrices of the workload through a Store-zechin plan and through
    the default (Ryser) plan: permanents/s of each, results compared exactly."""
    di = torch.from_numpy(np.ascontiguousarray(im).reshape(-1)).cuda()
    res = {}
    outs = {}
    for name, meth in (("store_zechin", lp.METHOD_SZ), ("ryser", lp.METHOD_AUTO)):
        o = torch.empty((count, 2), dtype=torch.int64, device="cuda")
        with lp.Plan(N, "u01", method=meth, max_batch=count) as p:
            p.batch(di, [N] * count, o, None, stream)
            torch.cuda.synchronize()
            ms = _event_ms(torch, stream, lambda: p.batch(di, [N] * count, o, None, stream))
        res[name + "_perm_per_s"] = count / (ms / 1000.0)
        outs[name] = o.cpu().numpy()
    res["identical"] = bool(np.array_equal(outs["store_zechin"], outs["ryser"]))
    return res


def measure_wide(lp, torch, stream):
    """Exact 0/1 permanents above 2^128 (PERM_FLAG_WIDE, Ryser modulo 2^192): one dense
    36 x 36 matrix with 14 zeros (the GPU tests check such matrices against the
    rook-number closed form)."""
    n = 36
    g = np.random.default_rng(3636)
    cells = set()
    while len(cells) < 14:
        cells.add((int(g.integers(n)), int(g.integers(n))))
    a = np.ones((n, n), dtype=np.int64)
    for i, j in cells:
        a[i, j] = 0
    d = torch.from_numpy(a.reshape(-1)).cuda()
    o = torch.empty(4, dtype=torch.int64, device="cuda")
    with lp.Plan(n, "u01", max_batch=1, flags=lp.FLAG_WIDE) as p:
        p.batch(d, [n], o, None, stream)
        torch.cuda.synchronize()
        ms = _event_ms(torch, stream, lambda: p.batch(d, [n], o, None, stream))
    value = lp.words_to_int(o.cpu().numpy())
    return {"n": n, "zeros": len(cells), "ms": ms, "bits": value.bit_length(),
            "codes_per_s": 2.0 ** n / (ms / 1000.0), "value": str(value)}


def measure_five_boson(lp, torch, stream, reps=20):
    """5-boson sampling: the 126 collision-free 5x5 submatrices of rows 0..4 of a
    9x9 Haar unitary and 100 Bernoulli(0.5) 5x5 0/1 matrices; latency of one call
    per method (CUDA events, median of `reps`), and all 126 amplitudes from one
    5x9 Store-zechin pass (perm_patterns)."""
    from paper_1802_02779_gb300 import workloads as wl
    cm, im = wl.five_boson()
    dc = torch.from_numpy(np.ascontiguousarray(cm).reshape(-1)).cuda()
    di = torch.from_numpy(np.ascontiguousarray(im).reshape(-1)).cuda()
    oc = torch.empty(len(cm), dtype=torch.complex128, device="cuda")
    oi = torch.empty((len(im), 2), dtype=torch.int64, device="cuda")
    u9 = torch.from_numpy(np.ascontiguousarray(wl.haar_unitary(9, wl.SEED_BASE + 1)[:5]).reshape(-1)).cuda()
    op = torch.empty(126, dtype=torch.complex128, device="cuda")

    def timed(fn, st=stream):
        ts = []
        for _ in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1000.0)
        return float(np.median(ts[2:]))

    res = {"complex": len(cm), "zero_one": len(im)}
    for name, meth in (("store_zechin", lp.METHOD_SZ), ("ryser", lp.METHOD_RYSER)):
        with lp.Plan(5, "c128", method=meth) as pc, lp.Plan(5, "u01", method=meth) as pi:
            res[name + "_complex_us"] = timed(lambda: pc.batch(dc, [5] * len(cm), oc, None, stream))
            res[name + "_zero_one_us"] = timed(lambda: pi.batch(di, [5] * len(im), oi, None, stream))
        # the same calls replayed as CUDA graphs (PERM_FLAG_GRAPH, which needs a non-default
        # stream; the graph is captured on the first call and the timing is the median after it)
        gs = torch.cuda.Stream()
        with lp.Plan(5, "c128", method=meth, flags=lp.FLAG_GRAPH) as pc, \
                lp.Plan(5, "u01", method=meth, flags=lp.FLAG_GRAPH) as pi:
            res[name + "_complex_graph_us"] = timed(lambda: pc.batch(dc, [5] * len(cm), oc, None, gs), gs)
            res[name + "_zero_one_graph_us"] = timed(lambda: pi.batch(di, [5] * len(im), oi, None, gs), gs)
    lib = lp.load()
    res["patterns_one_pass_us"] = timed(lambda: lib.perm_patterns(
        lp._VP(u9.data_ptr()), 1, 5, 9, lp._VP(op.data_ptr()), lp._VP(stream.cuda_stream)))
    return res


def measure_uneven(lp, torch, stream, count=20000):
    """Uneven-size batching: the whole stream of `count` requests (n uniform in
    8..28, 70% complex Haar submatrices, 30% 0/1 at density 0.3-0.7), each arm
    timed once over all of it: plain per-matrix launches, one batched call per
    dtype, and the same calls replayed as CUDA graphs (captured on a first call,
    then replayed)."""
    from paper_1802_02779_gb300 import workloads as wl
    reqs = wl.uneven_requests(count=count)
    groups = {}
    for dt in ("c128", "u01"):
        mats = [r.mat for r in reqs if r.dtype == dt]
        sizes = [m.shape[0] for m in mats]
        npdt = np.complex128 if dt == "c128" else np.int64
        flat = np.concatenate([np.ascontiguousarray(m, dtype=npdt).reshape(-1) for m in mats])
        dev = torch.from_numpy(flat).cuda()
        out = torch.empty((len(mats), 2), dtype=torch.float64 if dt == "c128" else torch.int64, device="cuda")
        groups[dt] = (sizes, dev, out)
    side = torch.cuda.Stream()
    res = {"requests": count, "n_range": [8, 28]}
    results = {}
    for name, flags in (("plain", lp.FLAG_PLAIN), ("batched", 0), ("graph", lp.FLAG_GRAPH)):
        plans = {dt: lp.Plan(28, dt, flags=flags, max_batch=count) for dt in groups}
        if name == "graph":                      # the capture call
            with torch.cuda.stream(side):
                for dt, (sizes, dev, out) in groups.items():
                    plans[dt].batch(dev, sizes, out, None, side)
            side.synchronize()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(side):
            for dt, (sizes, dev, out) in groups.items():
                plans[dt].batch(dev, sizes, out, None, side)
        side.synchronize()
        res[name + "_perm_per_s"] = count / (time.perf_counter() - t0)
        results[name] = {dt: g[2].cpu().numpy().copy() for dt, g in groups.items()}
        for p in plans.values():
            p.close()
    res["batched_vs_plain"] = res["batched_perm_per_s"] / res["plain_perm_per_s"]
    res["graph_vs_plain"] = res["graph_perm_per_s"] / res["plain_perm_per_s"]
    # the complex requests' Store-zechin work (the method's count, as the roofline) per second
    work = sum(sz_c128_standard_flops(r.n) for r in reqs if r.dtype == "c128")
    for name in ("plain", "batched", "graph"):
        res[name + "_complex_tflops"] = work * res[name + "_perm_per_s"] / count / 1e12
    res["same_bits"] = all((results["plain"][dt] == results[k][dt]).all()
                           for k in ("batched", "graph") for dt in groups)
    return res


def drive_server(srv, reqs, arrivals, limit_s, fifo=False):
    """Submit every request at its scheduled arrival (seconds after the start) and
    poll for completions.  fifo: poll in submission order and stop at the first
    request still pending (requests of one lane complete in order).  Returns the
    latencies (completion seen by perm_poll minus scheduled arrival), the orders
    of the completed requests and the time of the last completion."""
    pending = []
    lat, lat_n = [], []
    start = time.perf_counter()
    last = 0.0
    i = 0
    while i < len(reqs) or pending:
        now = time.perf_counter() - start
        submitted = False
        while i < len(reqs) and arrivals[i] <= now:
            pending.append((srv.submit(reqs[i].mat, reqs[i].dtype), arrivals[i], reqs[i].n))
            i += 1
            submitted = True
        rest = []
        for k, (t, t_arr, n) in enumerate(pending):
            state, _ = srv.poll(t)
            if state == "done":
                last = time.perf_counter() - start
                lat.append(last - t_arr)
                lat_n.append(n)
            else:
                rest.append((t, t_arr, n))
                if fifo:
                    rest.extend(pending[k + 1:])
                    break
        pending = rest
        if now > limit_s:
            break
        if not submitted:
            time.sleep(0.0002)
    return np.array(lat), np.array(lat_n), last


def pct(x, q):
    return float(np.percentile(x, q) * 1e3) if len(x) else None


def plain_rate(lp, reqs, limit_s):
    """Plain per-request launches: one blocking perm_batch_host call per request
    (PERM_FLAG_PLAIN plans, the default method choice), back to back."""
    plans = {}
    out = {"c128": np.zeros(2, dtype=np.float64), "u01": np.zeros(2, dtype=np.int64)}
    st = np.zeros(1, dtype=np.int32)
    lat = []
    try:
        start = time.perf_counter()
        for r in reqs:
            if r.dtype not in plans:
                plans[r.dtype] = lp.Plan(36, r.dtype, flags=lp.FLAG_PLAIN, max_batch=1)
            a = np.ascontiguousarray(r.mat, dtype=np.complex128 if r.dtype == "c128" else np.int64)
            t0 = time.perf_counter()
            plans[r.dtype].batch_host(a.reshape(-1), [a.shape[0]], out[r.dtype], st)
            lat.append(time.perf_counter() - t0)
            if time.perf_counter() - start > limit_s:
                break
        elapsed = time.perf_counter() - start
    finally:
        for p in plans.values():
            p.close()
    return len(lat) / elapsed, len(lat)


def measure_serving_n20(lp, count=4096, poisson_s=2.0):
    """The headline serving comparison: n = 20 complex requests (the batched
    workload's matrices) served by the server vs plain per-request launches.
    Saturated: all `count` requests submitted at once, permanents/s = count over
    the time to the last completion.  Plain: one blocking perm_batch_host per
    request (PERM_FLAG_PLAIN) on a sample.  Then Poisson arrivals at 0.8 x the
    saturated rate for `poisson_s` seconds: p50/p90/p99 latency."""
    from paper_1802_02779_gb300 import workloads as wl
    cm, _ = wl.batched_n20(count=count)
    reqs = [wl.Request(20, "c128", cm[i]) for i in range(count)]
    with lp.Server() as srv:
        drive_server(srv, reqs[:256], np.zeros(256), 60.0, fifo=True)          # warm-up
        lat, _, last = drive_server(srv, reqs, np.zeros(count), 120.0, fifo=True)
        served = count / last
        rate = 0.8 * served
        g = np.random.default_rng(wl.SEED_BASE + 10)
        arr = np.cumsum(g.exponential(1.0 / rate, size=int(rate * poisson_s * 1.2) + 16))
        arr = arr[arr < poisson_s]
        preqs = [reqs[k % count] for k in range(len(arr))]
        plat, _, plast = drive_server(srv, preqs, arr, poisson_s + 60.0, fifo=True)
    plain, nplain = plain_rate(lp, reqs[:256], 30.0)
    return {"requests": count, "served_perm_per_s": served, "plain_perm_per_s": plain,
            "served_vs_plain": served / plain, "plain_sample": nplain,
            "saturated_p50_ms": pct(lat, 50), "saturated_p99_ms": pct(lat, 99),
            "poisson": {"rate_per_s": rate, "requests": int(len(arr)), "completed": int(len(plat)),
                        "perm_per_s": float(len(plat) / plast) if plast else None,
                        "p50_ms": pct(plat, 50), "p90_ms": pct(plat, 90), "p99_ms": pct(plat, 99)},
            "how": "server: perm_submit / perm_poll from one host thread; plain: one blocking "
                   "perm_batch_host per request (PERM_FLAG_PLAIN)"}


def measure_serving(lp, requests=120, window_s=45.0):
    """The mixed serving workload: n uniform in 10..36, 70% complex Haar
    submatrices, 30% 0/1.  (1) Saturated: the first `requests` requests of the
    stream all submitted at once, served vs plain per-request launches on the same
    requests, permanents/s = requests over the time to the last completion.
    (2) Poisson arrivals for `window_s` seconds at 0.8 x the saturated served rate:
    latency = completion seen by perm_poll minus the scheduled arrival, and the
    same arrival trace through plain per-request calls."""
    from paper_1802_02779_gb300 import workloads as wl
    pool = wl.uneven_requests(count=2000, seed=wl.SEED_BASE + 8, n_lo=10, n_hi=36)
    sat = pool[:requests]
    with lp.Server() as srv:
        lat, lat_n, last = drive_server(srv, sat, np.zeros(len(sat)), 900.0)
        served = len(lat) / last
        rate = 0.8 * served
        g = np.random.default_rng(wl.SEED_BASE + 8)
        arrivals = np.cumsum(g.exponential(1.0 / rate, size=len(pool)))
        arrivals = arrivals[arrivals < window_s]
        preqs = pool[requests:requests + len(arrivals)]
        plat, plat_n, plast = drive_server(srv, preqs, arrivals, window_s + 120.0)
    plain_sat, _ = plain_rate(lp, sat, 900.0)
    plain = serve_plain(lp, preqs, arrivals, window_s + 120.0)
    return {"n_range": [10, 36], "table_budget": "server default (min(100 GB, 40% of free))",
            "saturated": {"requests": len(sat), "served_perm_per_s": served, "plain_perm_per_s": plain_sat,
                          "served_vs_plain": served / plain_sat,
                          "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99)},
            "poisson": {"arrival_rate_per_s": rate, "requests": int(len(preqs)), "completed": int(len(plat)),
                        "perm_per_s": float(len(plat) / plast) if plast else None,
                        "p50_ms": pct(plat, 50), "p90_ms": pct(plat, 90), "p99_ms": pct(plat, 99),
                        **latency_split(plat, plat_n), "plain": plain}}


def latency_split(lat, ns):
    """p90 of all requests, and p50/p99 of the small (n <= 20) and large requests apart."""
    out = {"p90_ms": float(np.percentile(lat, 90) * 1e3) if len(lat) else None}
    for name, sel in (("small_n_le_20", ns <= 20), ("large", ns > 20)):
        x = lat[sel]
        out[name] = {"count": int(len(x)),
                     "p50_ms": float(np.percentile(x, 50) * 1e3) if len(x) else None,
                     "p99_ms": float(np.percentile(x, 99) * 1e3) if len(x) else None}
    return out


def serve_plain(lp, reqs, arrivals, limit_s):
    """The same arrival trace served by plain per-request launches: one blocking
    perm_batch_host call per request in arrival order (PERM_FLAG_PLAIN plans,
    the default method choice), latency = completion minus scheduled arrival."""
    plans = {dt: lp.Plan(36, dt, flags=lp.FLAG_PLAIN, max_batch=1) for dt in ("c128", "u01")}
    out_c = np.zeros(2, dtype=np.float64)
    out_i = np.zeros(2, dtype=np.int64)
    st = np.zeros(1, dtype=np.int32)
    lat, lat_n = [], []
    try:
        start = time.perf_counter()
        for r, t_arr in zip(reqs, arrivals):
            now = time.perf_counter() - start
            if t_arr > now:
                time.sleep(t_arr - now)
            a = np.ascontiguousarray(r.mat, dtype=np.complex128 if r.dtype == "c128" else np.int64)
            plans[r.dtype].batch_host(a.reshape(-1), [a.shape[0]], out_c if r.dtype == "c128" else out_i, st)
            lat.append(time.perf_counter() - start - t_arr)
            lat_n.append(r.n)
            if time.perf_counter() - start > limit_s:
                break
        elapsed = time.perf_counter() - start
    finally:
        for p in plans.values():
            p.close()
    lat = np.array(lat)
    return {"completed": int(len(lat)),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
            "perm_per_s": float(len(lat) / elapsed) if len(lat) else 0.0,
            **latency_split(lat, np.array(lat_n)),
            "how": "one blocking perm_batch_host call per request in arrival order, PERM_FLAG_PLAIN"}


def run_single(args):
    """One matrix of order n through one method, timed twice (the second run reported)."""
    import torch
    from paper_1802_02779_gb300 import build, libperm as lp, workloads as wl
    build.build()
    if args.dtype == "c128":
        a = wl.gaussian_complex(args.n, wl.SEED_BASE + 5, scale=1.0 / args.n)
        dev = torch.from_numpy(a.reshape(-1)).cuda()
        out = torch.empty(1, dtype=torch.complex128, device="cuda")
    else:
        if args.dtype == "u01":
            a = wl.bernoulli01(1, args.n, 0.5, wl.SEED_BASE + 4)[0]
        else:   # small integers 0..2
            a = np.random.default_rng(wl.SEED_BASE + 4).integers(0, 3, (args.n, args.n)).astype(np.int64)
        dev = torch.from_numpy(a.reshape(-1)).cuda()
        out = torch.empty((1, 2), dtype=torch.int64, device="cuda")
    meth = lp.METHOD_SZ if args.method == "sz" else lp.METHOD_RYSER
    stream = torch.cuda.current_stream()
    times = []
    with lp.Plan(args.n, args.dtype, method=meth, max_batch=1) as p:
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.batch(dev, [args.n], out, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    print(json.dumps({"case": "single", "n": args.n, "method": args.method, "dtype": args.dtype,
                      "ms": times[-1], "value": str(out.cpu().numpy().tolist())}))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.case == "single":
        run_single(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
